// Persistent, length-bucketed batched kernel: the hot path.
//
// Work split.  The plan sorts pairs into classes by lane-group width G (32,
// 16, ..., 1; longest sweeps first) and, inside a class, by cost.  A warp
// takes one class at a time and splits into 32/G groups of G lanes.  Each
// group independently pulls a pair from its class queue, runs the forward
// sweep, then the reverse sweep of the same pair, then pulls the next pair,
// so groups never wait for one another's pairs.
//
// Sweep.  Lane t of a group holds query rows [t*R, t*R + R) of the current
// row strip in registers and walks the reference columns, lane t on column
// j = step - t: the anti-diagonal wavefront of ADEPT (Section II-B.2,
// Fig. 3) with R rows per lane.  The H and F values of the row above arrive
// by one register shuffle per value per step from lane t-1, executed by
// every lane alike, so the exchange never diverges (the lesson of GEVO's
// edits 5, 6, 8 and 10, Section VI-A).  Lane 0 takes them from the strip
// boundary instead: H = 0 / F = -infinity above the first strip (Section
// II-B.1's boundary row), and for later strips the last row of the previous
// strip, which lane G-1 wrote to global scratch.  Queries longer than G*R
// rows take several strips ("passes").  Residue codes and boundary words
// are loaded U steps before use.
//
// Every lane runs the same instruction stream on every step: columns outside
// a lane's range, idle groups and rows past the end of the query are
// computed with a pad residue whose scores are very negative, instead of
// being branched around.  Such cells never beat a real cell: their values
// come from real cells at an earlier column (or the same column and a
// smaller row) through non-positive steps, and ties go to the smaller
// column, then the smaller row.  Before a lane's first column the pad
// column leaves H = 0 and E = go, which gives the same first real column as
// the E = -infinity boundary.
//
// Recurrence (Section II-B.1, Fig. 8), per cell, six max-plus instructions:
//   E  = viaddmax(E, ge, Hg_left)          E = max(E + ge, H_left + go)
//   F  = viaddmax(F_up, ge, Hg_up)         F = max(F_up + ge, H_up + go)
//   T  = viaddmax(Hg_diag, s - go, E)      T = max(H_diag + s, E)
//   H  = vimax_relu(T, F)                  H = max(T, F, 0)
//   Hg = H + go
//   K  = viaddmax(H, 65535 - j, K)         end-cell key of the row
// Only Hg = H + go is stored per row; the profile holds s - go so the
// diagonal term needs no extra add.  All scores are scaled by 2^16, so
// K = (H << 16) | (65535 - j) orders cells by larger H, then smaller column,
// at one instruction per cell; rows are compared in ascending order with a
// strict "greater" so the smaller row wins ties.  The plan sends a pair
// here only when smax * min(n, m) <= 32766 and |go|, |ge| <= 16383, which
// keeps every scaled value and key inside int32.
//
// Reverse pass (Fig. 2(c)): the same sweep over the reversed prefixes
// a_qend..a_0 and b_rend..b_0.  Every 2U steps the group looks for a cell of
// score S; once found, it only finishes the columns up to that one.
#include "sw_internal.h"

namespace swgb {
namespace {

constexpr unsigned kFull = 0xffffffffu;
#ifndef SWGB_GROUP_UNROLL
#define SWGB_GROUP_UNROLL 4
#endif
constexpr int kU = SWGB_GROUP_UNROLL;  // steps per block; loads run one block ahead

// Sign-extended int8 byte B of w, moved to bits 16..31 (value << 16).
template <int B>
__device__ __forceinline__ int byte_hi(uint32_t w) {
    constexpr uint32_t sel = 0x44u | (uint32_t(B) << 8) | (uint32_t(B | 8) << 12);
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(w), "r"(0u), "r"(sel));
    return (int)d;
}

// Profile of one lane: for residue c in [0, A] (A = pad) and the lane's R
// rows, (s(q_row, c) - go) << 16, or a pad score for rows past the query.
// Layout [c][chunk][lane] of 16-byte chunks: conflict-free 128-bit loads
// whatever residue each lane asks for.
template <int R, bool P8>
__device__ __forceinline__ void build_profile(char *prof, int lane, const uint8_t *a, int dir,
                                              int row0, int nrows, const int8_t *smat, int A,
                                              int go) {
    int qa[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + r;
        qa[r] = i < nrows ? min((int)a[(ptrdiff_t)i * dir], A - 1) * A : -1;
    }
    for (int c = 0; c <= A; ++c) {
        if constexpr (P8) {
            static_assert(R == 16 || R == 8, "int8 profile holds 8 or 16 rows per lane");
            uint32_t w[R / 4];
#pragma unroll
            for (int k = 0; k < R / 4; ++k) w[k] = 0u;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int v = (qa[r] >= 0 && c < A) ? (int)smat[qa[r] + c] - go : -128;
                w[r >> 2] |= (uint32_t)(uint8_t)(int8_t)v << (8 * (r & 3));
            }
            if constexpr (R == 16)
                *reinterpret_cast<uint4 *>(prof + ((size_t)c * 32 + lane) * 16) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            else
                *reinterpret_cast<uint2 *>(prof + ((size_t)c * 32 + lane) * 8) =
                    make_uint2(w[0], w[1]);
        } else {
#pragma unroll
            for (int k = 0; k < R / 4; ++k) {
                int v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = 4 * k + u;
                    v[u] = (qa[r] >= 0 && c < A) ? ((int)smat[qa[r] + c] - go) * 65536
                                                 : kScaledPad;
                }
                *reinterpret_cast<int4 *>(prof + (((size_t)c * (R / 4) + k) * 32 + lane) * 16) =
                    make_int4(v[0], v[1], v[2], v[3]);
            }
        }
    }
}

template <int R, bool P8>
__device__ __forceinline__ void load_scores(const char *prof, int c, int lane, int (&sc)[R]) {
    if constexpr (P8) {
        uint32_t ws[R / 4];
        if constexpr (R == 16) {
            const uint4 w = *reinterpret_cast<const uint4 *>(prof + ((size_t)c * 32 + lane) * 16);
            ws[0] = w.x;
            ws[1] = w.y;
            ws[2] = w.z;
            ws[3] = w.w;
        } else {
            const uint2 w = *reinterpret_cast<const uint2 *>(prof + ((size_t)c * 32 + lane) * 8);
            ws[0] = w.x;
            ws[1] = w.y;
        }
#pragma unroll
        for (int k = 0; k < R / 4; ++k) {
            sc[4 * k + 0] = byte_hi<0>(ws[k]);
            sc[4 * k + 1] = byte_hi<1>(ws[k]);
            sc[4 * k + 2] = byte_hi<2>(ws[k]);
            sc[4 * k + 3] = byte_hi<3>(ws[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < R / 4; ++k) {
            const int4 v = *reinterpret_cast<const int4 *>(
                prof + (((size_t)c * (R / 4) + k) * 32 + lane) * 16);
            sc[4 * k + 0] = v.x;
            sc[4 * k + 1] = v.y;
            sc[4 * k + 2] = v.z;
            sc[4 * k + 3] = v.w;
        }
    }
}

// Per-lane bookkeeping of a group that only the strip and sweep transitions
// read: kept in shared memory (one array per field, indexed by thread) so
// the step loop's registers hold the DP state alone.
struct Cold {
    const uint8_t **a;   // row residues of the current sweep (a[i * dir])
    uint32_t **bnd;      // the pair's strip-boundary words
    int *n, *m, *passes, *ps, *target, *id, *S, *qend, *rend, *best_row;
    uint32_t *best_key;
};

constexpr int kColdWords = 2 * 2 + 11;  // 32-bit words per lane

}  // namespace

template <int R, bool P8>
__global__ void __launch_bounds__(kGroupWarps * 32, kGroupMinBlocks)
    sw_group_kernel(const __grid_constant__ GroupParams p) {
    extern __shared__ __align__(16) char smem_group[];
    const int A = p.alphabet;
    const int go = p.gap_open, ge = p.gap_extend;
    const int goS = go * 65536, geS = ge * 65536;
    constexpr int NT = kGroupWarps * 32;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const size_t prof_bytes = P8 ? (size_t)(A + 1) * 32 * R : (size_t)(A + 1) * (R / 4) * 32 * 16;
    int8_t *smat = reinterpret_cast<int8_t *>(smem_group);
    char *cold_base = smem_group + kMaxAlphabet * kMaxAlphabet;
    char *prof = cold_base + (size_t)kColdWords * 4 * NT + warp * prof_bytes;
    Cold cold;
    cold.a = reinterpret_cast<const uint8_t **>(cold_base);
    cold.bnd = reinterpret_cast<uint32_t **>(cold_base + 8 * NT);
    int *cw = reinterpret_cast<int *>(cold_base + 16 * NT);
    cold.n = cw;
    cold.m = cw + NT;
    cold.passes = cw + 2 * NT;
    cold.ps = cw + 3 * NT;
    cold.target = cw + 4 * NT;
    cold.id = cw + 5 * NT;
    cold.S = cw + 6 * NT;
    cold.qend = cw + 7 * NT;
    cold.rend = cw + 8 * NT;
    cold.best_row = cw + 9 * NT;
    cold.best_key = reinterpret_cast<uint32_t *>(cw + 10 * NT);
    for (int i = t; i < A * A; i += blockDim.x) smat[i] = p.mat[i];
    __syncthreads();

    // this warp starts on the class whose warp range holds it, then walks
    // the classes cyclically
    const int wid = blockIdx.x * kGroupWarps + warp;
    int start = 0;
    for (int c = 1; c < p.n_classes; ++c)
        if (wid >= p.classes[c].warp_begin) start = c;
    for (int visit = 0; visit < p.n_classes; ++visit) {
        const int cls = (start + visit) % p.n_classes;
        const ClassInfo ci = p.classes[cls];
        const int log2g = ci.log2g;
        const int G = 1 << log2g;
        const int gl = lane & (G - 1);
        const int gbase = lane & ~(G - 1);
        const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << gbase);

        // hot state: DP registers, the strip's step counters and pointers
        int H[R], E[R];
        uint32_t K[R];
        int diag0 = 0, outH = 0, outF = kScaledNegInf;
        int s = 0, lim = 0, stop = 0, dir = 1;
        const uint8_t *bcol = p.r;
        const uint32_t *bin = p.scratch;
        uint32_t *bout = p.scratch;
        bool has_in = false, has_out = false;
        bool live = false, rev = false, drained = false, reload = true;
        int cur_c[kU], nxt_c[kU];
        uint32_t cur_b[kU], nxt_b[kU];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            H[r] = 0;
            E[r] = kScaledNegInf;
            K[r] = 0u;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            cur_c[u] = nxt_c[u] = A;
            cur_b[u] = nxt_b[u] = 0u;
        }
        cold.id[t] = -1;

        // Starts strip ps of the current sweep: profile of this lane's rows,
        // fresh DP state, boundary buffers of the strip.
        auto begin_strip = [&](int ps) {
            const int n = cold.n[t], m = cold.m[t];
            build_profile<R, P8>(prof, lane, cold.a[t], dir, ps * G * R + gl * R, n, smat, A, go);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                H[r] = 0;
                E[r] = kScaledNegInf;
                K[r] = 0u;
            }
            diag0 = 0;
            outH = 0;
            outF = kScaledNegInf;
            s = 0;
            lim = stop + G - 1;
            uint32_t *bnd = cold.bnd[t];
            bin = bnd + ((ps + 1) & 1) * m;
            bout = bnd + (ps & 1) * m;
            has_in = ps > 0;
            has_out = ps + 1 < cold.passes[t];
            cold.ps[t] = ps;
            reload = true;
        };
        // Starts a sweep over (a, n) x (b, m) in direction d.
        auto begin_sweep = [&](const uint8_t *a, const uint8_t *b, int n, int m, int d) {
            cold.a[t] = a;
            bcol = b;
            dir = d;
            cold.n[t] = n;
            cold.m[t] = m;
            const int passes = (n > 0 && m > 0) ? (n + G * R - 1) / (G * R) : 0;
            cold.passes[t] = passes;
            cold.best_key[t] = 0u;
            cold.best_row[t] = 0x7fffffff;
            if (passes > 0) {
                stop = m;
                begin_strip(0);
            } else {
                stop = 0;
                s = 0;
                lim = 0;
                has_in = has_out = false;
                cold.ps[t] = 0;
            }
        };

        for (;;) {
            // ---- idle groups take the next pair of the class
            if (!live && !drained) {
                int idx = 0;
                if (gl == 0) idx = atomicAdd(p.counters + cls, 1);
                idx = __shfl_sync(gmask, idx, gbase);
                if (idx >= ci.count) {
                    drained = true;
                } else {
                    const PairInfo pi = p.pairs[ci.first + idx];
                    live = true;
                    rev = false;
                    cold.id[t] = pi.id;
                    cold.bnd[t] = p.scratch + (pi.scratch >= 0 ? pi.scratch : 0);
                    begin_sweep(p.q + pi.q, p.r + pi.r, pi.n, pi.m, 1);
                }
            }
            if (__all_sync(kFull, !live)) break;  // every group drained and idle

            const int mcols = live ? stop : 0;

            // ---- residue codes and boundary words: this block (if stale), next block
            if (reload) {
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int j = s + u - gl;
                    const bool in = (unsigned)j < (unsigned)mcols;
                    cur_c[u] = in ? min((int)bcol[(ptrdiff_t)j * dir], A - 1) : A;
                    cur_b[u] = (in && gl == 0 && has_in) ? bin[j] : 0u;
                }
                reload = false;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int j = s + kU + u - gl;
                const bool in = (unsigned)j < (unsigned)mcols;
                nxt_c[u] = in ? min((int)bcol[(ptrdiff_t)j * dir], A - 1) : A;
                nxt_b[u] = (in && gl == 0 && has_in) ? bin[j] : 0u;
            }

            // ---- U wavefront steps, the same instructions on every lane.  E and F
            // are held minus go, so the row-to-row chain is two instructions:
            //   F'_r = max(F'_{r-1} + ge, H_{r-1})        E'_r = max(E'_r + ge, H_left)
            //   T    = max(H_diag + (s - go), E'_r) + go  H_r  = max(F'_r + go, T, 0)
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int j = s + u - gl;
                const bool in = (unsigned)j < (unsigned)mcols;
                int inH = __shfl_up_sync(kFull, outH, 1, G);
                int inF = __shfl_up_sync(kFull, outF, 1, G);
                if (gl == 0) {
                    const bool from_bnd = in && has_in;
                    inH = from_bnd ? (int)(cur_b[u] << 16) : 0;
                    inF = from_bnd ? (int)(cur_b[u] & 0xFFFF0000u) : kScaledNegInf;
                }
                int c = in ? cur_c[u] : A;
                // tie this step's profile loads to its shuffle result, so the
                // compiler cannot hoist every unrolled step's loads (and their
                // registers) to the top of the block
                asm volatile("" : "+r"(c) : "r"(inH));
                int sc[R];
                load_scores<R, P8>(prof, c, lane, sc);
                const int cj = 65535 - max(j, 0);
                int diag = diag0;
                int F = __viaddmax_s32(inF, geS, inH);
                int hprev = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r > 0) F = __viaddmax_s32(F, geS, hprev);
                    E[r] = __viaddmax_s32(E[r], geS, H[r]);
                    const int T = __viaddmax_s32(diag, sc[r], E[r]) + goS;
                    const int h = __viaddmax_s32_relu(F, goS, T);
                    diag = H[r];
                    H[r] = h;
                    hprev = h;
                    K[r] = (uint32_t)__viaddmax_s32(h, cj, (int)K[r]);
                }
                outH = hprev;
                outF = F;
                if (in && has_out && gl == G - 1)
                    bout[j] = ((uint32_t)outH >> 16) | ((uint32_t)outF & 0xFFFF0000u);
                diag0 = inH;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                cur_c[u] = nxt_c[u];
                cur_b[u] = nxt_b[u];
            }
            s += kU;

            // ---- reverse sweep: stop once a cell of the forward score has appeared
            if (rev && live && ((s & (2 * kU - 1)) == 0)) {
                const int target = cold.target[t];
                uint32_t lk = K[0];
#pragma unroll
                for (int r = 1; r < R; ++r) lk = max(lk, K[r]);
                int found = (int)(lk >> 16) >= target ? 65535 - (int)(lk & 0xFFFFu) : 0x7fffffff;
                for (int off = 1; off < G; off <<= 1)
                    found = min(found, __shfl_xor_sync(gmask, found, off, G));
                if (found != 0x7fffffff && found + 1 < stop) {
                    stop = found + 1;
                    lim = stop + G - 1;
                }
            }

            // ---- end of a strip / sweep
            if (live && s >= lim) {
                const int ps = cold.ps[t], passes = cold.passes[t];
                uint32_t best_key = cold.best_key[t];
                int best_row = cold.best_row[t];
                if (ps < passes) {
                    const int row0 = ps * G * R + gl * R;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (K[r] > best_key) {
                            best_key = K[r];
                            best_row = row0 + r;
                        }
                }
                cold.best_key[t] = best_key;
                cold.best_row[t] = best_row;
                if (ps + 1 < passes) {
                    __syncwarp(gmask);  // boundary words written by lane G-1 -> lane 0
                    begin_strip(ps + 1);
                } else {
                    for (int off = 1; off < G; off <<= 1) {
                        const uint32_t ok = __shfl_xor_sync(gmask, best_key, off, G);
                        const int orow = __shfl_xor_sync(gmask, best_row, off, G);
                        if (ok > best_key || (ok == best_key && orow < best_row)) {
                            best_key = ok;
                            best_row = orow;
                        }
                    }
                    bool done = true;
                    if (!rev) {
                        const int S = (int)(best_key >> 16);
                        const int qend = best_row;
                        const int rend = 65535 - (int)(best_key & 0xFFFFu);
                        cold.S[t] = S;
                        if (S > 0) {
                            cold.qend[t] = qend;
                            cold.rend[t] = rend;
                            cold.target[t] = S;
                            rev = true;
                            done = false;
                            __syncwarp(gmask);
                            begin_sweep(cold.a[t] + qend, bcol + rend, qend + 1, rend + 1, -1);
                        }
                    }
                    if (done) {
                        if (gl == 0) {
                            const int S = cold.S[t];
                            const int id = cold.id[t];
                            int o0 = 0, o1 = -1, o2 = -1, o3 = -1, o4 = -1;
                            if (S > 0) {
                                const int qend = cold.qend[t], rend = cold.rend[t];
                                const int S2 = (int)(best_key >> 16);
                                const int l = 65535 - (int)(best_key & 0xFFFFu);
                                if (S2 != S) atomicOr(p.status, kStatusReverseMismatch);
                                o0 = S;
                                o1 = qend;
                                o2 = rend;
                                o3 = qend - best_row;
                                o4 = rend - l;
                            }
                            p.out.score[id] = o0;
                            p.out.qend[id] = o1;
                            p.out.rend[id] = o2;
                            p.out.qstart[id] = o3;
                            p.out.rstart[id] = o4;
                        }
                        live = false;
                        rev = false;
                        stop = 0;
                        __syncwarp(gmask);
                    }
                }
            }
        }
    }
}

size_t group_smem_bytes(ProfileKind kind, int alphabet) {
    const size_t per_warp = kind == ProfileKind::kInt8
                                ? (size_t)(alphabet + 1) * 32 * kRows
                                : (size_t)(alphabet + 1) * (kRows / 4) * 32 * 16;
    return kMaxAlphabet * kMaxAlphabet + (size_t)kColdWords * 4 * kGroupWarps * 32 +
           kGroupWarps * per_warp;
}

int group_blocks_per_sm(ProfileKind kind, int alphabet, int *smem_bytes) {
    const size_t smem = group_smem_bytes(kind, alphabet);
    if (smem_bytes) *smem_bytes = (int)smem;
    int blocks = 0;
    cudaError_t e;
    if (kind == ProfileKind::kInt8) {
        e = cudaFuncSetAttribute(sw_group_kernel<kRows, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &blocks, sw_group_kernel<kRows, true>, kGroupWarps * 32, smem);
    } else {
        e = cudaFuncSetAttribute(sw_group_kernel<kRows, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &blocks, sw_group_kernel<kRows, false>, kGroupWarps * 32, smem);
    }
    if (e != cudaSuccess) return -1;
    return blocks;
}

cudaError_t launch_group(const GroupParams &p, ProfileKind kind, int grid, cudaStream_t s) {
    if (p.n_classes <= 0 || grid <= 0) return cudaSuccess;
    const size_t smem = group_smem_bytes(kind, p.alphabet);
    if (kind == ProfileKind::kInt8)
        sw_group_kernel<kRows, true><<<grid, kGroupWarps * 32, smem, s>>>(p);
    else
        sw_group_kernel<kRows, false><<<grid, kGroupWarps * 32, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace swgb
