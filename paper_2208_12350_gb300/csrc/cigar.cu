// Traceback: the alignment itself, as a CIGAR, for pairs already located.
//
// The paper's method ends with a traceback from the maximal cell
// (Fig. 2(c)).  With the batched kernels' outputs (S, qend, rend, qstart,
// rstart) the alignment is the best global alignment of the located spans
// A' = a[qstart..qend] (N rows) and B' = b[rstart..rend] (M columns) under
// the same affine scoring; its score is S.  The global Gotoh recurrence
//   H[i][j] = max(H[i-1][j-1] + s, E[i][j], F[i][j])
//   E[i][j] = max(E[i][j-1] + ge, H[i][j-1] + go)
//   F[i][j] = max(F[i-1][j] + ge, H[i-1][j] + go)
// with H[0][j] = E[0][j] = go + (j-1) ge, H[i][0] = F[i][0] = go + (i-1) ge,
// H[0][0] = 0, is filled over the span recording per cell which terms won,
// and the walk back from (N, M) follows them: in state H it takes M if the
// diagonal won, else enters the gap state that won (E before F); in a gap
// state it emits D (E) or I (F) and returns to state H where the run
// opened.  The same rule, on the same values, as the CPU oracle.
//
// Fast path (spans of at most 512 rows whose values fit int32 with room):
// one lane group per pair, as in the batched kernel - lane t of a group of
// G lanes owns rows 16 t .. 16 t + 15 of the whole span (one strip) in
// registers and walks the columns on the anti-diagonal wavefront (lane t on
// column k - t + 1 at step k), taking the row above from lane t - 1 by a
// register shuffle.  Scores are int32 (the host checks the bound) and each
// cell's four decisions come from DPX max-with-predicate instructions
// (__vibmax_s32): E opened here, F opened here, E at least F, the diagonal
// at least both gaps.  They are packed as a nibble per row, one 64-bit word
// per lane and column, stored lane-major so that a group's stores of a step
// are G words.  Then the group's first lane walks back, reading one word
// per step while they are still in L2.  Pairs of a launch share a width G (the smallest power of
// two with 16 G >= N), 32 / G pairs per warp, longest first.
//
// General path (longer spans, or values beyond int32): one CTA of kThreads
// threads per pair; thread t owns row s*kThreads + t of row strip s and
// walks the columns on the anti-diagonal wavefront, taking the row above
// from thread t - 1 through shared memory (one barrier per step) and, for
// t = 0, from the previous strip's last row kept in global memory.  The
// choice bits of strip s are stored anti-diagonal by anti-diagonal, cell
// (t, column j) at byte (j + t) * kThreads + t of the strip, so each step's
// stores are one contiguous run.  Scores are int64: long spans with large
// gap costs reach values far below int32.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sw_internal.h"
#include "swgb.h"

namespace swgb {
namespace {

constexpr int kThreads = 128;
constexpr int64_t kNegInf64 = INT64_MIN / 4;
constexpr size_t kScratchBudget = size_t(1) << 30;  // choice bytes per launch

struct CigarPair {
    int64_t q, r;      // offsets of the spans' first residues
    int64_t tb;        // offset of the pair's choice bytes
    int64_t row;       // offset (int64 units) of its row buffer, 2 (M + 1)
    int64_t out;       // offset of its ops in the output
    int32_t N, M, id, pad;
};

struct CigarParams {
    const uint8_t *q, *r;
    const CigarPair *pairs;
    uint8_t *tb;
    int64_t *row;
    uint32_t *ops;
    int32_t *n_ops;
    int32_t A, go, ge;
    int8_t mat[kMaxAlphabet * kMaxAlphabet];
};

__host__ __device__ inline int64_t strips_of(int64_t N) { return (N + kThreads - 1) / kThreads; }
__host__ __device__ inline int64_t choice_bytes(int64_t N, int64_t M) {
    return strips_of(N) * (M + kThreads - 1) * kThreads;
}

__global__ void __launch_bounds__(kThreads) cigar_kernel(const __grid_constant__ CigarParams p) {
    __shared__ int smat[kMaxAlphabet * kMaxAlphabet];
    __shared__ int64_t upH[2][kThreads], upF[2][kThreads];
    const int A = p.A;
    const int64_t go = p.go, ge = p.ge;
    const int t = threadIdx.x;
    for (int i = t; i < A * A; i += kThreads) smat[i] = p.mat[i];
    const CigarPair cp = p.pairs[blockIdx.x];
    const int N = cp.N, M = cp.M;
    const uint8_t *qa = p.q + cp.q, *rb = p.r + cp.r;
    uint8_t *tb = p.tb + cp.tb;
    int64_t *rowH = p.row + cp.row, *rowF = rowH + (M + 1);
    for (int j = t; j <= M; j += kThreads) {
        rowH[j] = j == 0 ? 0 : go + (int64_t)(j - 1) * ge;
        rowF[j] = kNegInf64;
    }
    __syncthreads();

    const int64_t nstrips = strips_of(N);
    const int64_t sbytes = (int64_t)(M + kThreads - 1) * kThreads;
    for (int64_t s = 0; s < nstrips; ++s) {
        const int64_t i = s * kThreads + t + 1;  // 1-based row
        const bool valid = i <= N;
        const int x = valid ? min((int)qa[i - 1], A - 1) : 0;
        int64_t Hleft = go + (i - 1) * ge, Eleft = kNegInf64;
        int64_t Hdiag = i == 1 ? 0 : go + (i - 2) * ge;
        uint8_t *stb = tb + s * sbytes;
        for (int k = 0; k < M + kThreads - 1; ++k) {
            const int j = k - t + 1;  // 1-based column
            if (valid && j >= 1 && j <= M) {
                const int64_t Hup = t == 0 ? rowH[j] : upH[(k + 1) & 1][t - 1];
                const int64_t Fup = t == 0 ? rowF[j] : upF[(k + 1) & 1][t - 1];
                const int y = min((int)rb[j - 1], A - 1);
                const int64_t E = max(Eleft + ge, Hleft + go);
                const int64_t F = max(Fup + ge, Hup + go);
                const int64_t D = Hdiag + smat[x * A + y];
                const int64_t H = max(D, max(E, F));
                const int src = H == D ? 0 : (H == E ? 1 : 2);
                stb[(int64_t)k * kThreads + t] =
                    (uint8_t)(src | ((E == Hleft + go) << 2) | ((F == Hup + go) << 3));
                Hdiag = Hup;
                Hleft = H;
                Eleft = E;
                upH[k & 1][t] = H;
                upF[k & 1][t] = F;
                if (t == kThreads - 1) {  // last row of the strip, for the next one
                    rowH[j] = H;
                    rowF[j] = F;
                }
            }
            __syncthreads();
        }
    }

    if (t != 0) return;
    // walk back from (N, M) in state H; ops collected backwards, then reversed
    uint32_t *out = p.ops + cp.out;
    int nr = 0;
    auto push = [&](int op) {
        if (nr > 0 && (int)(out[nr - 1] & 15u) == op)
            out[nr - 1] += 16u;
        else
            out[nr++] = (1u << 4) | (uint32_t)op;
    };
    int i = N, j = M, state = 0;  // 0 = H, 1 = E, 2 = F
    const bool lin = p.go == p.ge;
    while (i > 0 || j > 0) {
        uint8_t c = 0;
        if (i > 0 && j > 0) {
            const int64_t s = (i - 1) / kThreads, tt = (i - 1) % kThreads;
            c = tb[s * sbytes + (int64_t)(j - 1 + tt) * kThreads + tt];
        }
        if (state == 0) {
            if (i > 0 && j > 0) {
                const int src = c & 3;
                if (src == 0) {
                    push(0);
                    --i;
                    --j;
                } else {
                    state = src;
                }
            } else {
                state = i == 0 ? 1 : 2;  // the boundary row is all D, the column all I
            }
        } else if (state == 1) {
            push(2);
            const bool open = (i > 0 && j > 0) ? ((c >> 2) & 1) != 0 : (j == 1 || lin);
            --j;
            if (open) state = 0;
        } else {
            push(1);
            const bool open = (i > 0 && j > 0) ? ((c >> 3) & 1) != 0 : (i == 1 || lin);
            --i;
            if (open) state = 0;
        }
    }
    for (int a = 0, b = nr - 1; a < b; ++a, --b) {
        const uint32_t tmp = out[a];
        out[a] = out[b];
        out[b] = tmp;
    }
    p.n_ops[cp.id] = nr;
}

// ---- fast path

constexpr int kTbRows = 16;        // rows per lane
constexpr int kTbMaxRows = 512;    // 32 lanes x 16 rows: one strip per span
constexpr int32_t kTbNegInf = -(1 << 29);

struct TbPair {
    int64_t q, r;   // offsets of the spans' first residues
    int64_t ch;     // offset (64-bit words) of its choice words: G x M of them
    int64_t out;    // offset of its ops in the output
    int32_t N, M, id, log2g;
};

struct TbParams {
    const uint8_t *q, *r;
    const TbPair *pairs;  // this launch's pairs (one width), longest first
    int32_t n_pairs;
    uint64_t *choice;
    uint32_t *ops;
    int32_t *n_ops;
    int32_t A, go, ge;
    int8_t mat[kMaxAlphabet * kMaxAlphabet];
};

__device__ void tb_walk(const TbParams &p, const TbPair &tp);

template <int LOG2G>
__global__ void __launch_bounds__(128) tb_fill_kernel(const __grid_constant__ TbParams p) {
    constexpr int G = 1 << LOG2G;
    __shared__ int smat[kMaxAlphabet * kMaxAlphabet];  // s - go
    const int A = p.A, go = p.go, ge = p.ge;
    for (int i = threadIdx.x; i < A * A; i += blockDim.x) smat[i] = (int)p.mat[i] - go;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int pidx = ((int)blockIdx.x * 4 + (int)(threadIdx.x >> 5)) * (32 / G) + (lane >> LOG2G);
    const bool has = pidx < p.n_pairs;
    TbPair tp{};
    if (has) tp = p.pairs[pidx];
    const int N = has ? tp.N : 0, M = has ? tp.M : 0;
    const uint8_t *qa = p.q + tp.q, *rb = p.r + tp.r;
    // this lane's rows i = 16 gl + r + 1 (1-based): matrix row offsets and
    // the column-0 boundary (H = go + (i - 1) ge, kept as H + go; E = -inf)
    int xr[kTbRows], X[kTbRows], E[kTbRows];
#pragma unroll
    for (int r = 0; r < kTbRows; ++r) {
        const int i0 = gl * kTbRows + r;  // 0-based row
        xr[r] = i0 < N ? min((int)qa[i0], A - 1) * A : 0;
        X[r] = go + i0 * ge + go;
        E[r] = kTbNegInf;
    }
    // The first row's diagonal: the row above at the previous column.  Lane 0
    // starts from H[0][0] + go; every lane passes down, until its first
    // column, its last row's column-0 boundary (H[16 gl + 16][0] + go), which
    // the lane below takes as the diagonal of its first column.
    int diag0 = go;
    int outX = X[kTbRows - 1], outF = kTbNegInf;
    uint64_t *ch = p.choice + tp.ch + (int64_t)gl * M;
    // the warp runs until its longest pair is done (pairs sorted longest first)
    int steps = has ? M + G - 1 : 0;
    for (int off = 16; off > 0; off >>= 1) steps = max(steps, __shfl_xor_sync(0xffffffffu, steps, off));
    int y_next = M > 0 && gl == 0 ? min((int)rb[0], A - 1) : 0;
    for (int k = 0; k < steps; ++k) {
        const int j = k - gl + 1;  // 1-based column of this lane
        // the row above at column j: lane gl - 1's last row (its step k - 1),
        // or for lane 0 the boundary row H[0][j] = go + (j - 1) ge, F = -inf
        int upX = __shfl_up_sync(0xffffffffu, outX, 1, G);
        int upF = __shfl_up_sync(0xffffffffu, outF, 1, G);
        if (gl == 0) {
            upX = go + (j - 1) * ge + go;
            upF = kTbNegInf;
        }
        const int diag_first = diag0;  // the row above at column j - 1
        diag0 = upX;
        const bool in = j >= 1 && j <= M;
        const int y = y_next;
        // next column's residue, fetched a step ahead
        y_next = (j + 1 >= 1 && j + 1 <= M) ? min((int)rb[j], A - 1) : 0;
        if (in) {
            int diag = diag_first;
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int r = 0; r < kTbRows; ++r) {
                bool eo, fo, ef, dm;
                const int e = __vibmax_s32(X[r], E[r] + ge, &eo);  // E = max(H_left + go, E + ge)
                const int f = __vibmax_s32(upX, upF + ge, &fo);    // F = max(H_up + go, F_up + ge)
                const int m1 = __vibmax_s32(e, f, &ef);
                const int h = __vibmax_s32(diag + smat[xr[r] + y], m1, &dm);
                const uint32_t nib = (uint32_t)dm | ((uint32_t)ef << 1) | ((uint32_t)eo << 2) |
                                     ((uint32_t)fo << 3);
                if (r < 8)
                    lo |= nib << (4 * r);
                else
                    hi |= nib << (4 * (r - 8));
                diag = X[r];
                X[r] = h + go;
                E[r] = e;
                upX = X[r];
                upF = f;
            }
            ch[j - 1] = ((uint64_t)hi << 32) | lo;
            outX = upX;
            outF = upF;
        }
    }
    // the group's first lane walks back while its choice words are in L2 (the
    // warp barrier orders the other lanes' stores before its loads)
    __syncwarp();
    if (has && gl == 0) tb_walk(p, tp);
}

// The walk back of one fast-path pair from (N, M), reading its choice words.
__device__ void tb_walk(const TbParams &p, const TbPair &tp) {
    const uint64_t *ch = p.choice + tp.ch;
    uint32_t *out = p.ops + tp.out;
    const bool lin = p.go == p.ge;
    int nr = 0;
    auto push = [&](int op) {
        if (nr > 0 && (int)(out[nr - 1] & 15u) == op)
            out[nr - 1] += 16u;
        else
            out[nr++] = (1u << 4) | (uint32_t)op;
    };
    int i = tp.N, j = tp.M, state = 0;  // 0 = H, 1 = E, 2 = F
    while (i > 0 || j > 0) {
        uint32_t c = 0;
        if (i > 0 && j > 0) {
            const uint64_t w = ch[(int64_t)((i - 1) / kTbRows) * tp.M + (j - 1)];
            c = (uint32_t)(w >> (4 * ((i - 1) % kTbRows))) & 15u;
        }
        if (state == 0) {
            if (i > 0 && j > 0) {
                if (c & 1u) {
                    push(0);
                    --i;
                    --j;
                } else {
                    state = (c & 2u) ? 1 : 2;
                }
            } else {
                state = i == 0 ? 1 : 2;  // the boundary row is all D, the column all I
            }
        } else if (state == 1) {
            push(2);
            const bool open = (i > 0 && j > 0) ? (c & 4u) != 0 : (j == 1 || lin);
            --j;
            if (open) state = 0;
        } else {
            push(1);
            const bool open = (i > 0 && j > 0) ? (c & 8u) != 0 : (i == 1 || lin);
            --i;
            if (open) state = 0;
        }
    }
    for (int a = 0, b = nr - 1; a < b; ++a, --b) {
        const uint32_t tmp = out[a];
        out[a] = out[b];
        out[b] = tmp;
    }
    p.n_ops[tp.id] = nr;
}

using TbFill = void (*)(TbParams);
TbFill tb_fill_of(int log2g) {
    switch (log2g) {
        case 0: return tb_fill_kernel<0>;
        case 1: return tb_fill_kernel<1>;
        case 2: return tb_fill_kernel<2>;
        case 3: return tb_fill_kernel<3>;
        case 4: return tb_fill_kernel<4>;
        default: return tb_fill_kernel<5>;
    }
}

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" int sw_cigar_capacity(const int32_t *results, int32_t n_pairs, int64_t *offsets) {
    if (!results || !offsets || n_pairs < 0)
        return set_error(SW_EINVAL, "sw_cigar_capacity: bad argument");
    const int64_t n = n_pairs;
    offsets[0] = 0;
    for (int64_t p = 0; p < n; ++p) {
        const int32_t S = results[p], qe = results[n + p], re = results[2 * n + p],
                      qs = results[3 * n + p], rs = results[4 * n + p];
        const int64_t room = S > 0 ? (int64_t)(qe - qs + 1) + (re - rs + 1) : 0;
        offsets[p + 1] = offsets[p] + std::max<int64_t>(room, 0);
    }
    return SW_OK;
}

extern "C" int sw_traceback(sw_ctx *ctx, const uint8_t *q_seqs, const int64_t *q_offsets,
                            const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                            const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                            int32_t gap_extend, const int32_t *results,
                            const int64_t *cigar_offsets, uint32_t *out_ops, int32_t *out_n_ops,
                            void *stream) {
    if (!ctx) return set_error(SW_EINVAL, "sw_traceback: ctx is NULL");
    if (n_pairs < 0 || (n_pairs > 0 && (!q_offsets || !r_offsets || !results || !cigar_offsets ||
                                        !out_n_ops)))
        return set_error(SW_EINVAL, "sw_traceback: bad argument");
    if (n_pairs == 0) return SW_OK;
    std::string msg;
    int rc = check_batch(q_offsets, r_offsets, n_pairs, score_matrix, alphabet_size, gap_open,
                         gap_extend, nullptr, nullptr, nullptr, &msg);
    if (rc != SW_OK) return set_error(rc, ("sw_traceback: " + msg).c_str());
    const int64_t n = n_pairs;
    int smax = 0;
    for (int k = 0; k < alphabet_size * alphabet_size; ++k)
        smax = std::max(smax, std::abs((int)score_matrix[k]));
    // per-cell magnitude bound of the fast path's int32 values
    const int64_t unit = (int64_t)-gap_open - gap_extend + smax;
    char buf[160];
    std::vector<CigarPair> pairs;  // general path
    std::vector<TbPair> fast;
    fast.reserve((size_t)n);
    for (int64_t p = 0; p < n; ++p) {
        const int32_t S = results[p], qe = results[n + p], re = results[2 * n + p],
                      qs = results[3 * n + p], rs = results[4 * n + p];
        if (S <= 0) continue;
        const int64_t qn = q_offsets[p + 1] - q_offsets[p], rm = r_offsets[p + 1] - r_offsets[p];
        if (qs < 0 || qs > qe || qe >= qn || rs < 0 || rs > re || re >= rm) {
            snprintf(buf, sizeof buf, "sw_traceback: pair %lld has coordinates outside it",
                     (long long)p);
            return set_error(SW_ERANGE, buf);
        }
        const int32_t N = qe - qs + 1, M = re - rs + 1;
        if (cigar_offsets[p + 1] - cigar_offsets[p] < (int64_t)N + M) {
            snprintf(buf, sizeof buf, "sw_traceback: pair %lld needs %lld ops of room",
                     (long long)p, (long long)N + M);
            return set_error(SW_ERANGE, buf);
        }
        if (N <= kTbMaxRows && ((int64_t)N + M + 2) * unit <= ((int64_t)1 << 28)) {
            TbPair tp{};
            tp.q = q_offsets[p] + qs;
            tp.r = r_offsets[p] + rs;
            tp.N = N;
            tp.M = M;
            tp.id = (int32_t)p;
            tp.out = cigar_offsets[p];
            int lg = 0;
            while ((kTbRows << lg) < N) ++lg;
            tp.log2g = lg;
            fast.push_back(tp);
            continue;
        }
        CigarPair cp{};
        cp.q = q_offsets[p] + qs;
        cp.r = r_offsets[p] + rs;
        cp.N = N;
        cp.M = M;
        cp.id = (int32_t)p;
        cp.out = cigar_offsets[p];
        pairs.push_back(cp);
    }
    if ((!pairs.empty() || !fast.empty()) && (!q_seqs || !r_seqs || !out_ops))
        return set_error(SW_EINVAL, "sw_traceback: NULL device pointer");
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    const int dev = ctx_device(ctx);
    if (dev != dev_prev && cudaSetDevice(dev) != cudaSuccess)
        return set_error(SW_ECUDA, "sw_traceback: cudaSetDevice failed");
    struct Restore {
        int dev, prev;
        ~Restore() {
            if (dev != prev && prev >= 0) cudaSetDevice(prev);
        }
    } restore{dev, dev_prev};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(out_n_ops, 0, (size_t)n * sizeof(int32_t), s);
    if (e != cudaSuccess) return set_error(SW_ECUDA, "sw_traceback: memset failed");

    // ---- fast path: widths longest first within each, choice words per pair
    if (!fast.empty()) {
        {
            // by width, then longest first: a counting sort on (width, Mmax - M)
            // over the batch's range of span lengths
            int32_t mlo = INT32_MAX, mhi = 0;
            for (const TbPair &t : fast) {
                mlo = std::min(mlo, t.M);
                mhi = std::max(mhi, t.M);
            }
            const size_t span = (size_t)(mhi - mlo) + 1;
            std::vector<int32_t> count(6 * span + 1, 0);
            auto key = [&](const TbPair &t) { return (size_t)t.log2g * span + (size_t)(mhi - t.M); };
            for (const TbPair &t : fast) ++count[key(t) + 1];
            for (size_t k = 1; k < count.size(); ++k) count[k] += count[k - 1];
            std::vector<TbPair> sorted(fast.size());
            for (const TbPair &t : fast) sorted[(size_t)count[key(t)]++] = t;
            fast.swap(sorted);
        }
        int64_t words = 0;
        for (TbPair &tp : fast) {
            tp.ch = words;
            words += ((int64_t)1 << tp.log2g) * tp.M;
        }
        void *ws = nullptr;
        const size_t pair_bytes = (fast.size() * sizeof(TbPair) + 255) & ~(size_t)255;
        if ((rc = ctx_alloc_async(ctx, pair_bytes + (size_t)words * 8, s, &ws)) != SW_OK)
            return rc;
        TbPair *d_fast = static_cast<TbPair *>(ws);
        uint64_t *d_choice = reinterpret_cast<uint64_t *>(static_cast<unsigned char *>(ws) + pair_bytes);
        if ((rc = ctx_upload_async(ctx, d_fast, fast.data(), fast.size() * sizeof(TbPair), s)) !=
            SW_OK) {
            cudaFreeAsync(ws, s);
            return rc;
        }
        TbParams tp;
        std::memset(&tp, 0, sizeof tp);
        tp.q = q_seqs;
        tp.r = r_seqs;
        tp.choice = d_choice;
        tp.ops = out_ops;
        tp.n_ops = out_n_ops;
        tp.A = alphabet_size;
        tp.go = gap_open;
        tp.ge = gap_extend;
        std::memcpy(tp.mat, score_matrix, (size_t)alphabet_size * alphabet_size);
        for (size_t a = 0; e == cudaSuccess && a < fast.size();) {
            size_t b = a;
            while (b < fast.size() && fast[b].log2g == fast[a].log2g) ++b;
            const int lg = fast[a].log2g;
            const int64_t per_block = 4 * (32 >> lg);
            tp.pairs = d_fast + a;
            tp.n_pairs = (int32_t)(b - a);
            const int64_t blocks = ((int64_t)(b - a) + per_block - 1) / per_block;
            tb_fill_of(lg)<<<(unsigned)blocks, 128, 0, s>>>(tp);
            e = cudaGetLastError();
            a = b;
        }
        cudaFreeAsync(ws, s);  // stream-ordered: after the kernels that use it
        if (e != cudaSuccess)
            return set_error(SW_ECUDA, (std::string("sw_traceback: ") + cudaGetErrorString(e)).c_str());
    }

    // ---- general path: one CTA per pair, chunks whose choice bytes fit the budget
    if (pairs.empty()) return SW_OK;
    CigarParams prm;
    std::memset(&prm, 0, sizeof prm);
    prm.q = q_seqs;
    prm.r = r_seqs;
    prm.ops = out_ops;
    prm.n_ops = out_n_ops;
    prm.A = alphabet_size;
    prm.go = gap_open;
    prm.ge = gap_extend;
    std::memcpy(prm.mat, score_matrix, (size_t)alphabet_size * alphabet_size);
    int64_t biggest = 0;
    for (const CigarPair &cp : pairs) biggest = std::max(biggest, choice_bytes(cp.N, cp.M));
    const size_t tb_cap = std::max<size_t>(kScratchBudget, (size_t)biggest);
    size_t row_cap = 0;
    for (const CigarPair &cp : pairs) row_cap += 2 * ((size_t)cp.M + 1);
    // chunks: a chunk's pairs share the choice scratch, so the next chunk runs
    // after it in stream order; every record is laid out before the upload
    std::vector<std::pair<size_t, size_t>> chunks;
    {
        size_t first = 0;
        int64_t row_at = 0;
        while (first < pairs.size()) {
            size_t last = first;
            int64_t used = 0;
            while (last < pairs.size()) {
                const int64_t b = choice_bytes(pairs[last].N, pairs[last].M);
                if (last > first && used + b > (int64_t)tb_cap) break;
                pairs[last].tb = used;
                pairs[last].row = row_at;
                row_at += 2 * ((int64_t)pairs[last].M + 1);
                used += b;
                ++last;
            }
            chunks.emplace_back(first, last);
            first = last;
        }
    }
    const size_t pair_bytes = (pairs.size() * sizeof(CigarPair) + 255) & ~(size_t)255;
    const size_t row_bytes = (row_cap * sizeof(int64_t) + 255) & ~(size_t)255;
    void *ws = nullptr;
    if ((rc = ctx_alloc_async(ctx, pair_bytes + row_bytes + tb_cap, s, &ws)) != SW_OK) return rc;
    unsigned char *wb = static_cast<unsigned char *>(ws);
    CigarPair *d_pairs = reinterpret_cast<CigarPair *>(wb);
    prm.row = reinterpret_cast<int64_t *>(wb + pair_bytes);
    prm.tb = wb + pair_bytes + row_bytes;
    e = cudaMemcpyAsync(d_pairs, pairs.data(), pairs.size() * sizeof(CigarPair),
                        cudaMemcpyHostToDevice, s);
    for (size_t c = 0; e == cudaSuccess && c < chunks.size(); ++c) {
        prm.pairs = d_pairs + chunks[c].first;
        cigar_kernel<<<(unsigned)(chunks[c].second - chunks[c].first), kThreads, 0, s>>>(prm);
        e = cudaGetLastError();
    }
    cudaFreeAsync(ws, s);
    if (e != cudaSuccess)
        return set_error(SW_ECUDA, (std::string("sw_traceback: ") + cudaGetErrorString(e)).c_str());
    return SW_OK;
}
