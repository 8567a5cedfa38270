// Persistent, length-bucketed batched kernel: the hot path.
//
// Work split.  A warp takes a task of up to 32/G pairs from a device queue
// (the plan orders tasks longest first); each pair gets a group of G lanes
// (G = 1..32).  Lane t of a group holds query rows [t*R, t*R + R) of the
// current row strip in registers and walks the reference columns, lane t
// working on column j = step - t: the anti-diagonal wavefront of ADEPT
// (Section II-B.2, Fig. 3) with R rows per lane instead of one.  The values
// a lane needs from the strip above (H and F of the row above, at this and
// the previous column) arrive by one register shuffle per value per step
// from lane t-1, executed by every lane alike, so the exchange never
// diverges (the lesson of GEVO's edits 5, 6, 8 and 10, Section VI-A).  Lane
// 0 of a group takes them from the strip boundary instead: zero/-infinity
// above the first strip (Section II-B.1's boundary row), and for later
// strips the last row of the previous strip, which lane G-1 wrote to global
// scratch.  Queries longer than G*R rows take several strips ("passes").
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
// a_qend..a_0 and b_rend..b_0, run by the same group right after the
// forward pass.  It stops as soon as the column holding the first cell of
// score S has been completed by every lane.
//
// Rows past the end of the query use a pad score (<= 0 after the shift back
// by go): such cells never beat a real cell, since their values come from
// real cells at an earlier column or the same column and a smaller row.
// Columns outside [0, m) are skipped by the lanes they fall on.
#include "sw_internal.h"

namespace swgb {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct LaneJob {
    const uint8_t *a;  // row residues: a[i * a_step]
    const uint8_t *b;  // column residues: b[j * b_step]
    uint32_t *bnd;     // 2*m boundary words (used when n > G*R)
    int a_step, b_step;
    int n, m;
};

// Sign-extended int8 byte `sel` of `w`, moved to bits 16..31 (value << 16).
template <int B>
__device__ __forceinline__ int byte_hi(uint32_t w) {
    constexpr uint32_t sel = 0x44u | (uint32_t(B) << 8) | (uint32_t(B | 8) << 12);
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(w), "r"(0u), "r"(sel));
    return (int)d;
}

template <int R, bool P8>
__device__ __forceinline__ void build_profile(char *prof, int lane, const LaneJob &job, int row0,
                                              int nrows, const int8_t *smat, int A, int go) {
    int qa[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + r;
        qa[r] = i < nrows ? min((int)job.a[(ptrdiff_t)i * job.a_step], A - 1) * A : -1;
    }
    for (int c = 0; c < A; ++c) {
        if constexpr (P8) {
            static_assert(R == 16, "int8 profile holds 16 rows per lane");
            uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int v = qa[r] >= 0 ? (int)smat[qa[r] + c] - go : -128;
                w[r >> 2] |= (uint32_t)(uint8_t)(int8_t)v << (8 * (r & 3));
            }
            *reinterpret_cast<uint4 *>(prof + ((size_t)c * 32 + lane) * 16) =
                make_uint4(w[0], w[1], w[2], w[3]);
        } else {
#pragma unroll
            for (int k = 0; k < R / 4; ++k) {
                int v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = 4 * k + u;
                    v[u] = qa[r] >= 0 ? ((int)smat[qa[r] + c] - go) * 65536 : kScaledPad;
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
        const uint4 w = *reinterpret_cast<const uint4 *>(prof + ((size_t)c * 32 + lane) * 16);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
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

// One local-alignment sweep (all row strips) of each group's job.  Every
// lane of the warp must call it.  On return every lane of a group holds the
// group's best key (H << 16 | 65535 - j) and the row of that cell.  With
// REV, the sweep stops once a cell of score `target` has been found and its
// column completed.
template <int R, bool P8, bool REV>
__device__ void sweep(const LaneJob &job, int G, int gl, int lane, char *prof,
                      const int8_t *smat, int A, int go, int ge, int target,
                      uint32_t &out_key, int &out_row) {
    const int goS = go * 65536, geS = ge * 65536;
    const int rpp = G * R;
    const int passes = (job.n > 0 && job.m > 0) ? (job.n + rpp - 1) / rpp : 0;
    const int max_passes = (int)__reduce_max_sync(kFull, (unsigned)passes);
    int stop = job.m;
    uint32_t best_key = 0;
    int best_row = 0x7fffffff;
    for (int ps = 0; ps < max_passes; ++ps) {
        const bool live = ps < passes;
        const int row0 = ps * rpp + gl * R;
        build_profile<R, P8>(prof, lane, job, row0, live ? job.n : 0, smat, A, go);
        __syncwarp();
        int Hg[R], E[R];
        uint32_t K[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            Hg[r] = goS;
            E[r] = kScaledNegInf;
            K[r] = 0u;
        }
        int diag0 = goS, outHg = goS, outF = kScaledNegInf;
        int mcols = live ? stop : 0;
        const uint32_t *bin = job.bnd + ((ps + 1) & 1) * job.m;
        uint32_t *bout = job.bnd + (ps & 1) * job.m;
        const bool write_bnd = live && (ps + 1 < passes) && gl == G - 1;
        const bool read_bnd = live && ps > 0 && gl == 0;
        const int lim = mcols > 0 ? mcols + G - 1 : 0;
        const int max_steps = (int)__reduce_max_sync(kFull, (unsigned)lim);
        for (int s = 0; s < max_steps; ++s) {
            int inHg = __shfl_up_sync(kFull, outHg, 1, G);
            int inF = __shfl_up_sync(kFull, outF, 1, G);
            const int j = s - gl;
            const bool act = j >= 0 && j < mcols;
            if (gl == 0) {
                inHg = goS;
                inF = kScaledNegInf;
            }
            if (read_bnd && act) {
                const uint32_t v = bin[j];
                inHg = (int)(v << 16);
                inF = (int)(v & 0xFFFF0000u);
            }
            if (act) {
                const int c = min((int)job.b[(ptrdiff_t)j * job.b_step], A - 1);
                int sc[R];
                load_scores<R, P8>(prof, c, lane, sc);
                const int cj = 65535 - j;
                int diag = diag0;
                int F = __viaddmax_s32(inF, geS, inHg);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r > 0) F = __viaddmax_s32(F, geS, Hg[r - 1]);
                    E[r] = __viaddmax_s32(E[r], geS, Hg[r]);
                    const int T = __viaddmax_s32(diag, sc[r], E[r]);
                    const int h = __vimax_s32_relu(T, F);
                    diag = Hg[r];
                    Hg[r] = h + goS;
                    K[r] = (uint32_t)__viaddmax_s32(h, cj, (int)K[r]);
                }
                outHg = Hg[R - 1];
                outF = F;
                if (write_bnd) bout[j] = ((uint32_t)outHg >> 16) | ((uint32_t)outF & 0xFFFF0000u);
                diag0 = inHg;
            }
            if constexpr (REV) {
                if ((s & 7) == 7) {
                    uint32_t lk = K[0];
#pragma unroll
                    for (int r = 1; r < R; ++r) lk = max(lk, K[r]);
                    int found = live && (int)(lk >> 16) >= target ? 65535 - (int)(lk & 0xFFFFu)
                                                                  : 0x7fffffff;
                    for (int off = 1; off < G; off <<= 1)
                        found = min(found, __shfl_xor_sync(kFull, found, off, G));
                    if (found != 0x7fffffff && found + 1 < stop) stop = found + 1;
                    mcols = live ? stop : 0;
                    const bool done = s + 1 >= (mcols > 0 ? mcols + G - 1 : 0);
                    if (__all_sync(kFull, done)) break;
                }
            }
        }
        if (live) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (K[r] > best_key) {
                    best_key = K[r];
                    best_row = row0 + r;
                }
        }
        __syncwarp();  // boundary words and the profile are reused next pass
    }
    for (int off = 1; off < G; off <<= 1) {
        const uint32_t ok = __shfl_xor_sync(kFull, best_key, off, G);
        const int orow = __shfl_xor_sync(kFull, best_row, off, G);
        if (ok > best_key || (ok == best_key && orow < best_row)) {
            best_key = ok;
            best_row = orow;
        }
    }
    out_key = best_key;
    out_row = best_row;
}

template <bool P8>
__host__ __device__ constexpr size_t profile_bytes_per_warp(int A) {
    return P8 ? (size_t)A * 32 * 16 : (size_t)A * (kRows / 4) * 32 * 16;
}

template <int R, bool P8>
__global__ void __launch_bounds__(kGroupWarps * 32)
    sw_group_kernel(const __grid_constant__ GroupParams p) {
    extern __shared__ __align__(16) char smem_group[];
    const int A = p.alphabet;
    int8_t *smat = reinterpret_cast<int8_t *>(smem_group);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    char *prof = smem_group + kMaxAlphabet * kMaxAlphabet + warp * profile_bytes_per_warp<P8>(A);
    for (int i = threadIdx.x; i < A * A; i += blockDim.x) smat[i] = p.mat[i];
    __syncthreads();

    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(p.counter, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= p.n_tasks) break;
        const GroupTask task = p.tasks[t];
        const int log2g = task.log2g;
        const int G = 1 << log2g;
        const int gid = lane >> log2g, gl = lane & (G - 1);
        const bool gv = gid < task.count;
        PairInfo pi = {0, 0, -1, 0, 0, 0, 0};
        if (gv) pi = p.pairs[task.first + gid];
        LaneJob fwd;
        fwd.a = p.q + pi.q;
        fwd.b = p.r + pi.r;
        fwd.bnd = pi.scratch >= 0 ? p.scratch + pi.scratch : nullptr;
        fwd.a_step = 1;
        fwd.b_step = 1;
        fwd.n = pi.n;
        fwd.m = pi.m;
        uint32_t key;
        int row;
        sweep<R, P8, false>(fwd, G, gl, lane, prof, smat, A, p.gap_open, p.gap_extend, 0, key,
                            row);
        const int S = (int)(key >> 16);
        const int qend = row;
        const int rend = 65535 - (int)(key & 0xFFFFu);
        const bool need_rev = gv && S > 0;
        LaneJob rev = fwd;
        rev.a = need_rev ? fwd.a + qend : fwd.a;
        rev.b = need_rev ? fwd.b + rend : fwd.b;
        rev.a_step = -1;
        rev.b_step = -1;
        rev.n = need_rev ? qend + 1 : 0;
        rev.m = need_rev ? rend + 1 : 0;
        uint32_t key2;
        int row2;
        sweep<R, P8, true>(rev, G, gl, lane, prof, smat, A, p.gap_open, p.gap_extend, S, key2,
                           row2);
        if (gv && gl == 0) {
            int o0 = 0, o1 = -1, o2 = -1, o3 = -1, o4 = -1;
            if (S > 0) {
                const int S2 = (int)(key2 >> 16);
                const int l = 65535 - (int)(key2 & 0xFFFFu);
                if (S2 != S) atomicOr(p.status, kStatusReverseMismatch);
                o0 = S;
                o1 = qend;
                o2 = rend;
                o3 = qend - row2;
                o4 = rend - l;
            }
            p.out.score[pi.id] = o0;
            p.out.qend[pi.id] = o1;
            p.out.rend[pi.id] = o2;
            p.out.qstart[pi.id] = o3;
            p.out.rstart[pi.id] = o4;
        }
    }
}

}  // namespace

size_t group_smem_bytes(ProfileKind kind, int alphabet) {
    const size_t per_warp = kind == ProfileKind::kInt8 ? profile_bytes_per_warp<true>(alphabet)
                                                       : profile_bytes_per_warp<false>(alphabet);
    return kMaxAlphabet * kMaxAlphabet + kGroupWarps * per_warp;
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
    if (p.n_tasks <= 0 || grid <= 0) return cudaSuccess;
    const size_t smem = group_smem_bytes(kind, p.alphabet);
    if (kind == ProfileKind::kInt8)
        sw_group_kernel<kRows, true><<<grid, kGroupWarps * 32, smem, s>>>(p);
    else
        sw_group_kernel<kRows, false><<<grid, kGroupWarps * 32, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace swgb
