// Traceback: the alignment itself, as a CIGAR, for pairs already located.
//
// The paper's method ends with a traceback from the maximal cell
// (Fig. 2(c)).  With the batched kernels' outputs (S, qend, rend, qstart,
// rstart) the alignment is the best global alignment of the located spans
// A' = a[qstart..qend] (N rows) and B' = b[rstart..rend] (M columns) under
// the same affine scoring; its score is S.  This kernel fills the global
// Gotoh recurrence over the span and records, per cell, which term won:
//   H[i][j] = max(H[i-1][j-1] + s, E[i][j], F[i][j])    2 bits: M, E or F
//   E[i][j] = max(E[i][j-1] + ge, H[i][j-1] + go)         1 bit: opened here
//   F[i][j] = max(F[i-1][j] + ge, H[i-1][j] + go)         1 bit: opened here
// with H[0][j] = E[0][j] = go + (j-1) ge, H[i][0] = F[i][0] = go + (i-1) ge,
// H[0][0] = 0.  One thread then walks back from (N, M): in state H it takes
// M if the diagonal won, else enters the gap state that won (E before F);
// in a gap state it emits D (E) or I (F) and returns to state H where the
// run opened.  The same rule, on the same values, as the CPU oracle.
//
// One CTA of kThreads threads per pair; thread t owns row s*kThreads + t of
// row strip s and walks the columns on the anti-diagonal wavefront, taking
// the row above from thread t - 1 through shared memory (one barrier per
// step) and, for t = 0, from the previous strip's last row kept in global
// memory.  The choice bits of strip s are stored anti-diagonal by
// anti-diagonal, cell (t, column j) at byte (j + t) * kThreads + t of the
// strip, so each step's stores are one contiguous run.  Scores are int64:
// long spans with large gap costs reach values far below int32.
#include <cuda_runtime.h>

#include <algorithm>
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
    char buf[160];
    std::vector<CigarPair> pairs;
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
        CigarPair cp{};
        cp.q = q_offsets[p] + qs;
        cp.r = r_offsets[p] + rs;
        cp.N = qe - qs + 1;
        cp.M = re - rs + 1;
        cp.id = (int32_t)p;
        cp.out = cigar_offsets[p];
        if (cigar_offsets[p + 1] - cigar_offsets[p] < (int64_t)cp.N + cp.M) {
            snprintf(buf, sizeof buf, "sw_traceback: pair %lld needs %lld ops of room",
                     (long long)p, (long long)cp.N + cp.M);
            return set_error(SW_ERANGE, buf);
        }
        pairs.push_back(cp);
    }
    if (!pairs.empty() && (!q_seqs || !r_seqs || !out_ops))
        return set_error(SW_EINVAL, "sw_traceback: NULL device pointer");
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    const int dev = ctx_device(ctx);
    if (dev != dev_prev && cudaSetDevice(dev) != cudaSuccess)
        return set_error(SW_ECUDA, "sw_traceback: cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
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
    // chunks of pairs whose choice bytes fit the scratch budget (or one pair)
    int64_t biggest = 0;
    for (const CigarPair &cp : pairs) biggest = std::max(biggest, choice_bytes(cp.N, cp.M));
    uint8_t *d_tb = nullptr;
    int64_t *d_row = nullptr;
    CigarPair *d_pairs = nullptr;
    const size_t tb_cap = std::max<size_t>(kScratchBudget, (size_t)biggest);
    size_t row_cap = 0;
    for (const CigarPair &cp : pairs) row_cap += 2 * ((size_t)cp.M + 1);
    cudaError_t e = cudaMemsetAsync(out_n_ops, 0, (size_t)n * sizeof(int32_t), s);
    if (e == cudaSuccess && !pairs.empty()) {
        if (cudaMalloc(&d_tb, tb_cap) != cudaSuccess ||
            cudaMalloc(&d_row, row_cap * sizeof(int64_t)) != cudaSuccess ||
            cudaMalloc(&d_pairs, pairs.size() * sizeof(CigarPair)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d_tb);
            cudaFree(d_row);
            cudaFree(d_pairs);
            if (dev != dev_prev && dev_prev >= 0) cudaSetDevice(dev_prev);
            return set_error(SW_ENOMEM, "sw_traceback: scratch allocation failed");
        }
        size_t first = 0;
        int64_t row_at = 0;
        while (e == cudaSuccess && first < pairs.size()) {
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
            e = cudaMemcpyAsync(d_pairs + first, pairs.data() + first,
                                (last - first) * sizeof(CigarPair), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) {
                prm.pairs = d_pairs + first;
                prm.tb = d_tb;
                prm.row = d_row;
                cigar_kernel<<<(unsigned)(last - first), kThreads, 0, s>>>(prm);
                e = cudaGetLastError();
            }
            // the pageable copy of the next chunk's records must not overtake
            // this chunk's use of the scratch; stream order keeps it behind
            first = last;
        }
    }
    // whatever was enqueued must finish before its scratch is freed, also
    // after a failed enqueue further on
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = es;
    cudaFree(d_tb);
    cudaFree(d_row);
    cudaFree(d_pairs);
    if (dev != dev_prev && dev_prev >= 0) cudaSetDevice(dev_prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(SW_ECUDA, (std::string("sw_traceback: ") + cudaGetErrorString(e)).c_str());
    }
    return SW_OK;
}
