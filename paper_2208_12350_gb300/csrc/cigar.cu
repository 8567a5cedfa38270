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
// Fast path (spans of at most 512 rows whose values fit int32 with room and
// whose scores s - go fit a signed byte): one lane group per pair, as in the
// batched kernel - lane t of a group of G lanes owns rows R t .. R t + R - 1
// of the whole span (one strip) in registers, R = 10, 12, 14 or 16 chosen
// per span with G (the smallest G R >= N), and walks the columns on the
// anti-diagonal wavefront (lane t on column k - t + 1 at step k), taking the
// row above from lane t - 1 by a register shuffle and its scores from a
// per-lane profile in shared memory (one 16-byte load per step).  Scores are
// int32 and each cell's four decisions come from DPX max-with-predicate
// instructions (__vibmax_s32): E opened here, F opened here, E at least F,
// the diagonal at least both gaps.  They are packed as a nibble per row, one
// 64-bit word per lane and column, stored by wavefront step (a group's
// stores of a step are contiguous).  Then the whole group
// walks back while the words are in L2, taking each run of the walk (up to
// 16 cells per round) with one ballot.  All classes of (G, R) share one
// launch, widest first, longest first within a class.
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
#include <condition_variable>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
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

// Worker threads for the host preparation of large batches, started on
// first use and kept (waking a parked thread costs far less than starting
// one).  run(k, fn) calls fn(0) .. fn(k - 1), fn(0) on the calling thread,
// and returns when all are done; one run at a time.
#ifndef SWGB_TB_HOST_THREADS
#define SWGB_TB_HOST_THREADS 8
#endif
class HostPool {
  public:
    static constexpr int kMax = SWGB_TB_HOST_THREADS;
    static HostPool &get() {
        static HostPool *pool = new HostPool();  // never destroyed: parked threads end with the process
        return *pool;
    }
    void run(int k, const std::function<void(int)> &fn) {
        std::lock_guard<std::mutex> one(run_mu_);
        k = std::min(k, kMax);
        {
            std::unique_lock<std::mutex> lk(mu_);
            while ((int)th_.size() < k - 1) {
                const int id = (int)th_.size() + 1;
                th_.emplace_back([this, id] { loop(id); });
                th_.back().detach();
            }
            job_ = &fn;
            want_ = k;
            left_ = k - 1;
            ++gen_;
        }
        cv_.notify_all();
        fn(0);
        std::unique_lock<std::mutex> lk(mu_);
        done_.wait(lk, [this] { return left_ == 0; });
        job_ = nullptr;
    }

  private:
    void loop(int id) {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            cv_.wait(lk, [&] { return gen_ != seen; });
            seen = gen_;
            if (id >= want_) continue;
            const std::function<void(int)> *fn = job_;
            lk.unlock();
            (*fn)(id);
            lk.lock();
            if (--left_ == 0) done_.notify_one();
        }
    }
    std::mutex run_mu_, mu_;
    std::condition_variable cv_, done_;
    std::vector<std::thread> th_;
    const std::function<void(int)> *job_ = nullptr;
    uint64_t gen_ = 0;
    int want_ = 0, left_ = 0;
};

// ---- fast path

constexpr int kTbMaxRows = 512;  // 32 lanes x 16 rows: one strip per span
constexpr int kTbRowOpts = 4;    // rows per lane: 10, 12, 14 or 16
constexpr int32_t kTbNegInf = -(1 << 29);
// Fast path, the adds of a cell: 0 = plain adds; 1 = E + ge, F + ge and
// H_diag + s as multiply-adds by a one the compiler cannot see (FMA pipe);
// 2 = also H + go.
#ifndef SWGB_TB_FMA
#define SWGB_TB_FMA 0
#endif
// Fast path, cells of the current run the walk examines per round (at least;
// G when the group is wider).
#ifndef SWGB_TB_LOOKAHEAD
#define SWGB_TB_LOOKAHEAD 16
#endif
// Fast path, resident blocks per SM the fill kernel's registers are sized for.
#ifndef SWGB_TB_MIN_BLOCKS
#define SWGB_TB_MIN_BLOCKS 1
#endif
// Fast path, the choice nibbles: 1 = each decision ORs its bit in under its
// predicate; 0 = a nibble assembled from the four flags, then shifted in
// (measured on 100k DNA spans: 1 is 7 % faster end to end).
#ifndef SWGB_TB_PACK
#define SWGB_TB_PACK 1
#endif
__host__ __device__ constexpr int tb_rows(int ri) { return 10 + 2 * ri; }

struct TbPair {
    int64_t q, r;   // offsets of the spans' first residues
    int64_t ch;     // offset (64-bit words) of its choice words: G x (M + G - 1) of them
    int64_t out;    // offset of its ops in the output
    int32_t N, M, id, cls;  // cls = log2(G) * kTbRowOpts + rows option
};

constexpr int kTbClasses = 6 * kTbRowOpts;

// A launch's blocks by class: blocks [block0, next class's block0) take the
// class's pairs [first, first + count), 128 / G of them per block.
struct TbClassRange {
    int32_t cls, first, count, block0;
};

struct TbParams {
    const uint8_t *q, *r;
    const TbPair *pairs;  // by class (widest first), longest first within a class
    int32_t n_pairs;
    int32_t n_ranges;
    TbClassRange ranges[kTbClasses];
    uint64_t *choice;
    uint32_t *ops;
    int32_t *n_ops;
    int32_t A, go, ge;
    int8_t mat[kMaxAlphabet * kMaxAlphabet];
};

// The walk back of one pair from (N, M), by its whole lane group.  The walk
// is a sequence of runs - diagonal moves in state H, moves left in state E
// (D ops), moves up in state F (I ops) - and each round looks ahead along the
// current run: lane t of the group reads the choice nibbles of the next L
// cells t L .. t L + L - 1 of the run (G L >= 16 cells in all), a ballot
// finds the first cell that ends the run, and the whole run up to it is
// taken at once.  All lanes keep the same walk state; lane 0 writes the ops.
template <int LOG2G, int R>
__device__ __forceinline__ void tb_walk_group(const TbParams &p, const TbPair &tp, int gl) {
    constexpr int G = 1 << LOG2G;
    constexpr int L = G >= SWGB_TB_LOOKAHEAD ? 1 : SWGB_TB_LOOKAHEAD / G;  // cells per lane and round
    constexpr int T = G * L;                 // cells per round
    const int lane = threadIdx.x & 31;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int gshift = lane & ~(G - 1);
    const uint64_t *ch = p.choice + tp.ch;
    uint32_t *out = p.ops + tp.out;
    const int M = tp.M;
    const bool lin = p.go == p.ge;
    auto cell = [&](int ii, int jj) -> uint32_t {  // 1 <= ii <= N, 1 <= jj <= M
        const int l = (ii - 1) / R, r = ii - 1 - l * R;
        return (uint32_t)(ch[(int64_t)(jj - 1 + l) * G + l] >> (4 * r)) & 15u;
    };
    int nr = 0, run_op = -1, run_len = 0;
    auto push = [&](int op, int len) {
        if (op == run_op) {
            run_len += len;
            return;
        }
        if (run_len > 0) {
            if (gl == 0) out[nr] = ((uint32_t)run_len << 4) | (uint32_t)run_op;
            ++nr;
        }
        run_op = op;
        run_len = len;
    };
    int i = tp.N, j = M, state = 0;  // 0 = H, 1 = E, 2 = F
    while (i > 0 || j > 0) {
        // this lane's first cell of the round that ends the run (T: none), and
        // what that cell says (16: the run reached the matrix edge)
        int stop = T;
        uint32_t cs = 0;
#pragma unroll
        for (int u = 0; u < L; ++u) {
            const int t = gl * L + u;
            if (stop < T) break;
            if (state == 0) {
                const int ii = i - t, jj = j - t;
                if (ii < 1 || jj < 1) {
                    stop = t;
                    cs = 16;
                } else {
                    const uint32_t c = cell(ii, jj);
                    if (!(c & 1u)) {
                        stop = t;
                        cs = c;
                    }
                }
            } else if (state == 1) {
                // a D at (i, j - t), then the gap opened there?
                const int jj = j - t;
                if (jj < 1) {
                    stop = t;  // (not reached: a gap opens at column 1 at the latest)
                    cs = 16;
                } else if (i > 0 ? (cell(i, jj) & 4u) != 0 : (jj == 1 || lin)) {
                    stop = t;
                }
            } else {
                const int ii = i - t;
                if (ii < 1) {
                    stop = t;
                    cs = 16;
                } else if (j > 0 ? (cell(ii, j) & 8u) != 0 : (ii == 1 || lin)) {
                    stop = t;
                }
            }
        }
        const unsigned m = __ballot_sync(gmask, stop < T) >> gshift;
        const int src = m ? __ffs(m) - 1 : 0;
        const int first = __shfl_sync(gmask, stop, src + gshift);
        const uint32_t c0 = __shfl_sync(gmask, cs, src + gshift);
        if (state == 0) {
            if (!m) {
                push(0, T);
                i -= T;
                j -= T;
            } else {
                if (first > 0) push(0, first);
                i -= first;
                j -= first;
                if (c0 == 16)
                    state = i == 0 ? 1 : 2;  // the boundary row is all D, the column all I
                else
                    state = (c0 & 2u) ? 1 : 2;
                if (i == 0 && j == 0) break;
            }
        } else if (state == 1) {
            const int len = m ? first + 1 : T;
            push(2, len);
            j -= len;
            if (m) state = 0;
        } else {
            const int len = m ? first + 1 : T;
            push(1, len);
            i -= len;
            if (m) state = 0;
        }
    }
    if (run_len > 0) {
        if (gl == 0) out[nr] = ((uint32_t)run_len << 4) | (uint32_t)run_op;
        ++nr;
    }
    // the ops were produced last first: reverse them, the group together
    __syncwarp(gmask);
    for (int a = gl; a < nr / 2; a += G) {
        const uint32_t x = out[a], y = out[nr - 1 - a];
        out[a] = y;
        out[nr - 1 - a] = x;
    }
    if (gl == 0) p.n_ops[tp.id] = nr;
}

// One lane group of G lanes per pair; lane t owns rows R t .. R t + R - 1 of
// the span.  Each lane's scores s - go for its rows come from a profile it
// builds in shared memory (R bytes per residue code, one 16-byte load per
// step), so a step reads no per-cell table entry.
template <int LOG2G, int R>
__device__ __forceinline__ void tb_fill(const TbParams &p, const TbClassRange &cr,
                                        const int *smat, uint4 *tb_prof) {
    constexpr int G = 1 << LOG2G;
    static_assert(R <= 16, "a lane's decisions fill at most one 64-bit word per column");
    const int A = p.A, go = p.go, ge = p.ge;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int grp = (int)threadIdx.x >> LOG2G;
    const int pidx = ((int)blockIdx.x - cr.block0) * (128 / G) + grp;
    const bool has = pidx < cr.count;
    TbPair tp{};
    if (has) tp = p.pairs[cr.first + pidx];
    const int N = has ? tp.N : 0, M = has ? tp.M : 0;
    const uint8_t *qa = p.q + tp.q, *rb = p.r + tp.r;
    [[maybe_unused]] const int one = (int)(blockDim.x >> 7);  // 1: blocks have 128 threads
    {
        // this lane's profile: byte r of entry y is s(q[R gl + r], y) - go (the
        // host checks that it fits a signed byte); rows past the span take 0
        int xr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i0 = gl * R + r;
            xr[r] = i0 < N ? min((int)qa[i0], A - 1) * A : -1;
        }
        for (int y = 0; y < A; ++y) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (xr[r] >= 0) w[r >> 2] |= ((uint32_t)smat[xr[r] + y] & 0xFFu) << (8 * (r & 3));
            tb_prof[y * 128 + threadIdx.x] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    // this lane's rows i = R gl + r + 1 (1-based): the column-0 boundary
    // (H = go + (i - 1) ge, kept as H + go; E = -inf)
    int X[R], E[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i0 = gl * R + r;  // 0-based row
        X[r] = go + i0 * ge + go;
        E[r] = kTbNegInf;
    }
    // The first row's diagonal: the row above at the previous column.  Lane 0
    // starts from H[0][0] + go; every lane passes down, until its first
    // column, its last row's column-0 boundary (H[R gl + R][0] + go), which
    // the lane below takes as the diagonal of its first column.
    int diag0 = go;
    int outX = X[R - 1], outF = kTbNegInf;
    // choice words by step: lane l's word for column j sits at step j - 1 + l,
    // so the G words a group stores at a step are contiguous
    uint64_t *ch = p.choice + tp.ch + gl;
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
            const uint4 pw = tb_prof[y * 128 + threadIdx.x];
            const uint32_t pws[4] = {pw.x, pw.y, pw.z, pw.w};
            int diag = diag_first;
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                // byte r & 3 of word r >> 2 with its sign replicated into the
                // upper bytes (PTX prmt: a selector nibble with its top bit set
                // replicates the sign of the byte it names)
                constexpr unsigned kSx[4] = {0x8880u, 0x9991u, 0xAAA2u, 0xBBB3u};
                uint32_t sx;
                asm("prmt.b32 %0, %1, 0, %2;" : "=r"(sx) : "r"(pws[r >> 2]), "r"(kSx[r & 3]));
                const int sc = (int)sx;
                bool eo, fo, ef, dm;
                int e_in, f_in, d_in;
                if constexpr (SWGB_TB_FMA >= 1) {
                    // the adds as multiply-adds by a one the compiler cannot
                    // see, so that they issue on the FMA pipe
                    asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(e_in) : "r"(E[r]), "r"(one), "r"(ge));
                    asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(f_in) : "r"(upF), "r"(one), "r"(ge));
                    asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(d_in) : "r"(diag), "r"(one), "r"(sc));
                } else {
                    e_in = E[r] + ge;
                    f_in = upF + ge;
                    d_in = diag + sc;
                }
                const int e = __vibmax_s32(X[r], e_in, &eo);  // E = max(H_left + go, E + ge)
                const int f = __vibmax_s32(upX, f_in, &fo);   // F = max(H_up + go, F_up + ge)
                const int m1 = __vibmax_s32(e, f, &ef);
                const int h = __vibmax_s32(d_in, m1, &dm);
#if SWGB_TB_PACK
                // each decision sets its bit by a predicated or
                uint32_t &wd = r < 8 ? lo : hi;
                const int sh = 4 * (r & 7);
                if (dm) wd |= 1u << sh;
                if (ef) wd |= 2u << sh;
                if (eo) wd |= 4u << sh;
                if (fo) wd |= 8u << sh;
#else
                const uint32_t nib = (uint32_t)dm | ((uint32_t)ef << 1) | ((uint32_t)eo << 2) |
                                     ((uint32_t)fo << 3);
                if (r < 8)
                    lo |= nib << (4 * r);
                else
                    hi |= nib << (4 * (r - 8));
#endif
                diag = X[r];
                if constexpr (SWGB_TB_FMA >= 2)
                    asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(X[r]) : "r"(h), "r"(one), "r"(go));
                else
                    X[r] = h + go;
                E[r] = e;
                upX = X[r];
                upF = f;
            }
            ch[(int64_t)k * G] = ((uint64_t)hi << 32) | lo;
            outX = upX;
            outF = upF;
        }
    }
    // the group walks back while its choice words are in L2 (the barrier
    // orders every lane's stores before the loads)
    __syncwarp();
    if (has) tb_walk_group<LOG2G, R>(p, tp, gl);
}

// Every fast-path pair of a call in one launch: each block finds its class
// (lane-group width and rows per lane) in the range table and runs that
// instantiation, so the classes share one grid and one tail.
__global__ void __launch_bounds__(128, SWGB_TB_MIN_BLOCKS) tb_fill_kernel(const __grid_constant__ TbParams p) {
    extern __shared__ uint4 tb_prof[];                 // [code][thread]: R bytes of s - go
    __shared__ int smat[kMaxAlphabet * kMaxAlphabet];  // s - go
    const int A = p.A;
    for (int i = threadIdx.x; i < A * A; i += blockDim.x) smat[i] = (int)p.mat[i] - p.go;
    __syncthreads();
    int c = 0;
    for (int k = 1; k < p.n_ranges; ++k)
        if ((int)blockIdx.x >= p.ranges[k].block0) c = k;
    const TbClassRange cr = p.ranges[c];
#define SWGB_TB_CASE(LG, RI)                                               \
    case (LG) * kTbRowOpts + (RI):                                         \
        tb_fill<LG, tb_rows(RI)>(p, cr, smat, tb_prof);                    \
        break;
#define SWGB_TB_ROWS(LG) \
    SWGB_TB_CASE(LG, 0) SWGB_TB_CASE(LG, 1) SWGB_TB_CASE(LG, 2) SWGB_TB_CASE(LG, 3)
    switch (cr.cls) {
        SWGB_TB_ROWS(0)
        SWGB_TB_ROWS(1)
        SWGB_TB_ROWS(2)
        SWGB_TB_ROWS(3)
        SWGB_TB_ROWS(4)
        SWGB_TB_ROWS(5)
        default: break;
    }
#undef SWGB_TB_ROWS
#undef SWGB_TB_CASE
}

// The width and rows per lane of a span of N rows: the smallest G R >= N over
// R in {10, 12, 14, 16} and G a power of two up to 32 (ties: more rows per
// lane, so fewer lanes and less skew).
__host__ __device__ int tb_class_of(int32_t N) {
    int best = -1, best_rows = INT32_MAX;
    for (int ri = kTbRowOpts - 1; ri >= 0; --ri) {
        int lg = 0;
        while ((tb_rows(ri) << lg) < N && lg < 5) ++lg;
        const int rows = tb_rows(ri) << lg;
        if (rows >= N && rows < best_rows) {
            best_rows = rows;
            best = lg * kTbRowOpts + ri;
        }
    }
    return best;
}

// tb_class_of for N in [1, kTbMaxRows], from a table built once
int tb_class(int32_t N) {
    struct Table {
        int8_t cls[kTbMaxRows + 1];
        Table() {
            for (int k = 0; k <= kTbMaxRows; ++k) cls[k] = (int8_t)tb_class_of(k);
        }
    };
    static const Table t;
    return t.cls[N];
}


// The fast path's one launch over records already on the device, classes
// widest first; d_choice holds the choice words the records' offsets name.
cudaError_t launch_tb_fill(const TbPair *d_fast, int32_t n_fast, uint64_t *d_choice,
                           const TbClassRange *ranges, int n_ranges, int64_t blocks,
                           const uint8_t *q, const uint8_t *r, uint32_t *ops, int32_t *n_ops,
                           const int8_t *mat, int A, int go, int ge, cudaStream_t s) {
    TbParams tp;
    std::memset(&tp, 0, sizeof tp);
    tp.q = q;
    tp.r = r;
    tp.choice = d_choice;
    tp.ops = ops;
    tp.n_ops = n_ops;
    tp.A = A;
    tp.go = go;
    tp.ge = ge;
    std::memcpy(tp.mat, mat, (size_t)A * A);
    tp.pairs = d_fast;
    tp.n_pairs = n_fast;
    tp.n_ranges = n_ranges;
    std::memcpy(tp.ranges, ranges, sizeof(TbClassRange) * (size_t)n_ranges);
    // each thread's profile: one 16-byte entry per residue code; with the
    // kernel's static shared memory (the score table) the block can pass the
    // default 48 KB
    const size_t prof_bytes = (size_t)A * 128 * 16;
    cudaError_t e = cudaFuncSetAttribute(tb_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)prof_bytes);
    if (e != cudaSuccess) return e;
    tb_fill_kernel<<<(unsigned)blocks, 128, prof_bytes, s>>>(tp);
    return cudaGetLastError();
}

// The general path for `pairs` (their q, r, N, M, id and out set): one CTA
// per pair, in chunks whose choice bytes fit the scratch budget.
int run_general(sw_ctx *ctx, std::vector<CigarPair> &pairs, const uint8_t *q_seqs,
                const uint8_t *r_seqs, uint32_t *out_ops, int32_t *out_n_ops,
                const int8_t *score_matrix, int alphabet_size, int gap_open, int gap_extend,
                cudaStream_t s, const char *who) {
    int rc = SW_OK;
    cudaError_t e = cudaSuccess;
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
        return set_error(SW_ECUDA, (std::string(who) + ": " + cudaGetErrorString(e)).c_str());
    return SW_OK;
}


// ---- the preparation on the device (sw_traceback_device)
//
// The same classification as the host's, as three kernels over results and
// offsets already on the device: a histogram of the fast-path pairs over
// (class, span-length bucket) slots with the choice words each slot needs,
// one block's exclusive scan of the slots (record and word positions, and
// the class ranges), and a scatter that writes each pair's record at its
// slot's next position, its choice words at the slot's next word offset.
// Within a slot pairs land in arbitrary order; each pair's ops depend on its
// own span alone.
constexpr int kTbMShift = 3;     // span-length buckets of 8 columns
constexpr int kTbMBuckets = 512;  // per class; spans of 4,088 columns or more share the last
constexpr int kTbSlots = kTbClasses * kTbMBuckets;
constexpr int kTbScanThreads = 1024;
static_assert(kTbSlots % kTbScanThreads == 0, "whole slots per scan thread");

struct TbDevSummary {
    unsigned long long err;  // ~(pair << 3 | kind) of the first bad pair (atomicMax), 0: none
    long long words;         // choice words of the fast path
    int32_t n_fast, n_general, n_ranges, blocks;
    TbClassRange ranges[kTbClasses];
};

struct TbDevArgs {
    const int64_t *qo, *ro, *co;
    const int32_t *res;
    int64_t n;
    int64_t unit;   // per-cell magnitude bound of the fast path's values
    int bytes_ok;   // every s - go fits a signed byte
    uint32_t *slot_count;
    unsigned long long *slot_words;
    uint32_t *slot_pos;
    unsigned long long *slot_wpos;
    TbPair *records;
    CigarPair *general;
    TbDevSummary *sum;
};

// kind: -1 bad (bad = 1 coordinates outside the pair, 2 too little op room,
// 3 offsets negative or decreasing, 4 a length above SW_MAX_LEN), 0 nothing
// to trace (score 0), 1 fast path, 2 general path
struct TbDevClass {
    int kind, bad, slot, cls;
    int32_t N, M, qs, rs;
    int64_t wpp;
};

__device__ TbDevClass tb_dev_class(const TbDevArgs &a, int64_t p) {
    TbDevClass c{};
    const int64_t q0 = a.qo[p], r0 = a.ro[p];
    const int64_t qn = a.qo[p + 1] - q0, rm = a.ro[p + 1] - r0;
    if (q0 < 0 || r0 < 0 || qn < 0 || rm < 0 || qn > SW_MAX_LEN || rm > SW_MAX_LEN) {
        c.kind = -1;
        c.bad = (qn > SW_MAX_LEN || rm > SW_MAX_LEN) && qn >= 0 && rm >= 0 && q0 >= 0 && r0 >= 0 ? 4 : 3;
        return c;
    }
    const int64_t n = a.n;
    const int32_t S = a.res[p], qe = a.res[n + p], re = a.res[2 * n + p], qs = a.res[3 * n + p],
                  rs = a.res[4 * n + p];
    if (S <= 0) return c;
    if (qs < 0 || qs > qe || qe >= qn || rs < 0 || rs > re || re >= rm) {
        c.kind = -1;
        c.bad = 1;
        return c;
    }
    c.N = qe - qs + 1;
    c.M = re - rs + 1;
    c.qs = qs;
    c.rs = rs;
    if (a.co[p + 1] - a.co[p] < (int64_t)c.N + c.M) {
        c.kind = -1;
        c.bad = 2;
        return c;
    }
    if (a.bytes_ok && c.N <= kTbMaxRows && ((int64_t)kTbMaxRows + c.M + 2) * a.unit <= ((int64_t)1 << 28)) {
        c.kind = 1;
        c.cls = tb_class_of(c.N);
        const int64_t G = (int64_t)1 << (c.cls / kTbRowOpts);
        c.wpp = G * (c.M + G - 1);
        // widest class first, longest span first within a class
        c.slot = (kTbClasses - 1 - c.cls) * kTbMBuckets +
                 (kTbMBuckets - 1 - min(c.M >> kTbMShift, kTbMBuckets - 1));
        return c;
    }
    c.kind = 2;
    return c;
}

__global__ void tb_dev_classify(const __grid_constant__ TbDevArgs a) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const TbDevClass c = tb_dev_class(a, p);
        if (c.kind < 0) {
            atomicMax(&a.sum->err, ~(((unsigned long long)p << 3) | (unsigned long long)c.bad));
        } else if (c.kind == 1) {
            atomicAdd(a.slot_count + c.slot, 1u);
            atomicAdd(a.slot_words + c.slot, (unsigned long long)c.wpp);
        } else if (c.kind == 2) {
            const int g = atomicAdd(&a.sum->n_general, 1);
            CigarPair cp{};
            cp.q = a.qo[p] + c.qs;
            cp.r = a.ro[p] + c.rs;
            cp.N = c.N;
            cp.M = c.M;
            cp.id = (int32_t)p;
            cp.out = a.co[p];
            a.general[g] = cp;
        }
    }
}

// One block: exclusive scans of the slot counts and words, then the class
// ranges (classes widest first) and the fill's blocks per class.
__global__ void __launch_bounds__(kTbScanThreads) tb_dev_scan(const __grid_constant__ TbDevArgs a) {
    constexpr int per = kTbSlots / kTbScanThreads;
    __shared__ uint32_t wc[32];
    __shared__ unsigned long long ww[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, k0 = t * per;
    uint32_t c = 0;
    unsigned long long w = 0;
    for (int i = 0; i < per; ++i) {
        c += a.slot_count[k0 + i];
        w += a.slot_words[k0 + i];
    }
    uint32_t ic = c;
    unsigned long long iw = w;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t oc = __shfl_up_sync(0xffffffffu, ic, off);
        const unsigned long long ow = __shfl_up_sync(0xffffffffu, iw, off);
        if (lane >= off) {
            ic += oc;
            iw += ow;
        }
    }
    if (lane == 31) {
        wc[warp] = ic;
        ww[warp] = iw;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t x = wc[lane];
        unsigned long long y = ww[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t ox = __shfl_up_sync(0xffffffffu, x, off);
            const unsigned long long oy = __shfl_up_sync(0xffffffffu, y, off);
            if (lane >= off) {
                x += ox;
                y += oy;
            }
        }
        wc[lane] = x;
        ww[lane] = y;
    }
    __syncthreads();
    uint32_t bc = (warp ? wc[warp - 1] : 0u) + ic - c;
    unsigned long long bw = (warp ? ww[warp - 1] : 0ull) + iw - w;
    for (int i = 0; i < per; ++i) {
        a.slot_pos[k0 + i] = bc;
        a.slot_wpos[k0 + i] = bw;
        bc += a.slot_count[k0 + i];
        bw += a.slot_words[k0 + i];
    }
    __syncthreads();  // every thread's slot positions are visible to thread 0
    if (t == 0) {
        const uint32_t total = wc[31];
        int nr = 0;
        int64_t blocks = 0;
        for (int k = 0; k < kTbClasses; ++k) {
            const uint32_t first = a.slot_pos[k * kTbMBuckets];
            const uint32_t end = k + 1 < kTbClasses ? a.slot_pos[(k + 1) * kTbMBuckets] : total;
            if (end > first) {
                const int cls = kTbClasses - 1 - k;
                const int per_block = 128 >> (cls / kTbRowOpts);
                a.sum->ranges[nr] = TbClassRange{cls, (int32_t)first, (int32_t)(end - first),
                                                 (int32_t)blocks};
                blocks += (end - first + per_block - 1) / per_block;
                ++nr;
            }
        }
        a.sum->n_fast = (int32_t)total;
        a.sum->words = (long long)ww[31];
        a.sum->n_ranges = nr;
        a.sum->blocks = (int32_t)blocks;
    }
}

__global__ void tb_dev_scatter(const __grid_constant__ TbDevArgs a) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const TbDevClass c = tb_dev_class(a, p);
        if (c.kind != 1) continue;
        const uint32_t pos = atomicAdd(a.slot_pos + c.slot, 1u);
        const unsigned long long wpos = atomicAdd(a.slot_wpos + c.slot, (unsigned long long)c.wpp);
        TbPair tp;
        tp.q = a.qo[p] + c.qs;
        tp.r = a.ro[p] + c.rs;
        tp.ch = (int64_t)wpos;
        tp.out = a.co[p];
        tp.N = c.N;
        tp.M = c.M;
        tp.id = (int32_t)p;
        tp.cls = c.cls;
        a.records[pos] = tp;
    }
}

// Room per pair ((qend - qstart + 1) + (rend - rstart + 1) ops for an
// aligned pair, 0 otherwise) and its exclusive scan, by one block over tiles
// of its width; offsets[n] ends as the total.
constexpr int kCapThreads = 1024;
__global__ void __launch_bounds__(kCapThreads) cigar_capacity_kernel(const int32_t *res, int64_t n,
                                                                    int64_t *offsets) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += kCapThreads) {
        const int64_t p = base + t;
        long long room = 0;
        if (p < n && res[p] > 0)
            room = (long long)(res[n + p] - res[3 * n + p] + 1) + (res[2 * n + p] - res[4 * n + p] + 1);
        room = room > 0 ? room : 0;
        long long inc = room;
        for (int off = 1; off < 32; off <<= 1) {
            const long long o = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += o;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            long long x = wsum[lane];
            for (int off = 1; off < 32; off <<= 1) {
                const long long o = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += o;
            }
            wsum[lane] = x;
        }
        __syncthreads();
        const long long c0 = carry;
        if (p < n) offsets[p] = c0 + (warp ? wsum[warp - 1] : 0) + inc - room;
        __syncthreads();
        if (t == 0) carry = c0 + wsum[31];
        __syncthreads();
    }
    if (t == 0) offsets[n] = carry;
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
    // scoring checks here; the offsets are checked pair by pair below
    int rc = check_batch(q_offsets, r_offsets, 0, score_matrix, alphabet_size, gap_open,
                         gap_extend, nullptr, nullptr, nullptr, &msg);
    if (rc != SW_OK) return set_error(rc, ("sw_traceback: " + msg).c_str());
    const int64_t n = n_pairs;
    int smax = 0;
    for (int k = 0; k < alphabet_size * alphabet_size; ++k)
        smax = std::max(smax, std::abs((int)score_matrix[k]));
    // per-cell magnitude bound of the fast path's int32 values, and its
    // profile of s - go as signed bytes
    const int64_t unit = (int64_t)-gap_open - gap_extend + smax;
    bool bytes_ok = true;
    for (int k = 0; k < alphabet_size * alphabet_size; ++k) {
        const int v = (int)score_matrix[k] - gap_open;
        bytes_ok = bytes_ok && v >= -128 && v <= 127;
    }
    char buf[160];
    // The pairs are split over up to 8 host threads (large batches): each
    // classifies its share - a key per fast-path pair (class and span
    // length; kNoKey for the others, kept per thread across calls so that its
    // pages stay mapped), a histogram of the keys, its general-path pairs -
    // and later writes its fast-path records in sorted order.
    constexpr uint32_t kNoKey = 0xFFFFFFFFu;
    thread_local std::vector<uint32_t> keyv_store;
    keyv_store.resize((size_t)n);
    uint32_t *const keyv = keyv_store.data();  // (the worker threads have stores of their own)
    const int n_thr = (int)std::max<int64_t>(
        1, std::min<int64_t>({HostPool::kMax, (int64_t)std::thread::hardware_concurrency(),
                              n / 4096}));
    struct Share {
        int64_t begin = 0, end = 0, n_fast = 0, bad = -1;
        // 1: coordinates outside the pair, 2: too little op room, 3: offsets
        // negative or decreasing, 4: a length above SW_MAX_LEN
        int bad_kind = 0;
        int32_t mlo = INT32_MAX, mhi = 0;
        std::vector<CigarPair> general;
        std::vector<int32_t> hist;  // per key slot (second pass)
    };
    std::vector<Share> sh((size_t)n_thr);
    for (int t = 0; t < n_thr; ++t) {
        sh[t].begin = n * t / n_thr;
        sh[t].end = n * (t + 1) / n_thr;
    }
    auto run_shares = [&](auto &&fn) {
        if (n_thr == 1) {
            fn(sh[0]);
            return;
        }
        HostPool::get().run(n_thr, [&](int t) { fn(sh[t]); });
    };
    run_shares([&](Share &w) {
        for (int64_t p = w.begin; p < w.end; ++p) {
            keyv[p] = kNoKey;
            const int64_t qn = q_offsets[p + 1] - q_offsets[p], rm = r_offsets[p + 1] - r_offsets[p];
            if (q_offsets[p] < 0 || r_offsets[p] < 0 || qn < 0 || rm < 0 || qn > SW_MAX_LEN ||
                rm > SW_MAX_LEN) {
                w.bad = p;
                w.bad_kind = (qn > SW_MAX_LEN || rm > SW_MAX_LEN) && qn >= 0 && rm >= 0 &&
                                     q_offsets[p] >= 0 && r_offsets[p] >= 0
                                 ? 4
                                 : 3;
                return;
            }
            const int32_t S = results[p], qe = results[n + p], re = results[2 * n + p],
                          qs = results[3 * n + p], rs = results[4 * n + p];
            if (S <= 0) continue;
            if (qs < 0 || qs > qe || qe >= qn || rs < 0 || rs > re || re >= rm) {
                w.bad = p;
                w.bad_kind = 1;
                return;
            }
            const int32_t N = qe - qs + 1, M = re - rs + 1;
            if (cigar_offsets[p + 1] - cigar_offsets[p] < (int64_t)N + M) {
                w.bad = p;
                w.bad_kind = 2;
                return;
            }
            if (bytes_ok && N <= kTbMaxRows &&
                ((int64_t)kTbMaxRows + M + 2) * unit <= ((int64_t)1 << 28)) {
                keyv[p] = ((uint32_t)tb_class(N) << 16) | (uint32_t)M;  // M < 2^16
                ++w.n_fast;
                w.mlo = std::min(w.mlo, M);
                w.mhi = std::max(w.mhi, M);
                continue;
            }
            CigarPair cp{};
            cp.q = q_offsets[p] + qs;
            cp.r = r_offsets[p] + rs;
            cp.N = N;
            cp.M = M;
            cp.id = (int32_t)p;
            cp.out = cigar_offsets[p];
            w.general.push_back(cp);
        }
    });
    std::vector<CigarPair> pairs;  // general path
    int64_t n_fast = 0;
    int32_t mlo = INT32_MAX, mhi = 0;
    for (const Share &w : sh) {
        if (w.bad >= 0) {
            const int64_t p = w.bad;
            if (w.bad_kind == 3)
                snprintf(buf, sizeof buf,
                         "sw_traceback: offsets of pair %lld negative or decreasing", (long long)p);
            else if (w.bad_kind == 4)
                snprintf(buf, sizeof buf, "sw_traceback: pair %lld has a length above SW_MAX_LEN",
                         (long long)p);
            else if (w.bad_kind == 1)
                snprintf(buf, sizeof buf, "sw_traceback: pair %lld has coordinates outside it",
                         (long long)p);
            else
                snprintf(buf, sizeof buf, "sw_traceback: pair %lld needs %lld ops of room",
                         (long long)p,
                         (long long)(results[n + p] - results[3 * n + p] + 1) +
                             (results[2 * n + p] - results[4 * n + p] + 1));
            return set_error(SW_ERANGE, buf);
        }
        n_fast += w.n_fast;
        mlo = std::min(mlo, w.mlo);
        mhi = std::max(mhi, w.mhi);
        pairs.insert(pairs.end(), w.general.begin(), w.general.end());
    }
    if ((!pairs.empty() || n_fast > 0) && (!q_seqs || !r_seqs || !out_ops))
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

    // ---- fast path: classes widest first, longest first within each (a
    // counting sort on (class, Mmax - M)), the records written in that order
    // straight into the page-locked staging buffer
    if (n_fast > 0) {
        const size_t span = (size_t)(mhi - mlo) + 1;
        const size_t n_slots = (size_t)kTbClasses * span;
        auto slot = [&](uint32_t k) {
            return (size_t)(kTbClasses - 1 - (int)(k >> 16)) * span + (size_t)(mhi - (int32_t)(k & 0xFFFFu));
        };
        run_shares([&](Share &w) {
            w.hist.assign(n_slots, 0);
            for (int64_t p = w.begin; p < w.end; ++p)
                if (keyv[p] != kNoKey) ++w.hist[slot(keyv[p])];
        });
        // stable counting sort: slot-major, then share, then pair order.  A
        // slot fixes the class and M, so its pairs' choice words (G M each)
        // follow from its first position; the classes' ranges from the slots
        std::vector<int64_t> slot_first(n_slots), slot_words(n_slots);
        TbClassRange ranges[kTbClasses];
        int n_ranges = 0;
        int64_t blocks = 0, words = 0;
        {
            int64_t at = 0;
            for (size_t k = 0; k < n_slots; ++k) {
                const int cls = kTbClasses - 1 - (int)(k / span);
                const int64_t G = (int64_t)1 << (cls / kTbRowOpts);
                const int64_t wpp = G * (mhi - (int64_t)(k % span) + G - 1);
                slot_first[k] = at;
                slot_words[k] = words;
                const int64_t at0 = at;
                for (Share &w : sh) {
                    const int32_t c = w.hist[k];
                    w.hist[k] = (int32_t)at;
                    at += c;
                }
                words += (at - at0) * wpp;
                if (at > at0) {
                    if (n_ranges == 0 || ranges[n_ranges - 1].cls != cls)
                        ranges[n_ranges++] = {cls, (int32_t)at0, 0, 0};
                    ranges[n_ranges - 1].count += (int32_t)(at - at0);
                }
            }
            for (int c = 0; c < n_ranges; ++c) {
                const int64_t per_block = 128 >> (ranges[c].cls / kTbRowOpts);
                ranges[c].block0 = (int32_t)blocks;
                blocks += (ranges[c].count + per_block - 1) / per_block;
            }
        }
        const size_t rec_bytes = (size_t)n_fast * sizeof(TbPair);
        void *host = nullptr;
        if ((rc = ctx_pinned_acquire(ctx, rec_bytes, &host)) != SW_OK) return rc;
        TbPair *fast = static_cast<TbPair *>(host);
        run_shares([&](Share &w) {
            for (int64_t p = w.begin; p < w.end; ++p) {
                const uint32_t k = keyv[p];
                if (k == kNoKey) continue;
                const size_t sl = slot(k);
                const int64_t pos = w.hist[sl]++;
                TbPair &tp = fast[pos];
                const int32_t qe = results[n + p], re = results[2 * n + p],
                              qs = results[3 * n + p], rs = results[4 * n + p];
                tp.q = q_offsets[p] + qs;
                tp.r = r_offsets[p] + rs;
                tp.out = cigar_offsets[p];
                tp.N = qe - qs + 1;
                tp.M = re - rs + 1;
                tp.id = (int32_t)p;
                tp.cls = (int32_t)(k >> 16);
                const int64_t G = (int64_t)1 << (tp.cls / kTbRowOpts);
                tp.ch = slot_words[sl] + (pos - slot_first[sl]) * G * (tp.M + G - 1);
            }
        });
        void *ws = nullptr;
        const size_t pair_bytes = (rec_bytes + 255) & ~(size_t)255;
        if ((rc = ctx_alloc_async(ctx, pair_bytes + (size_t)words * 8, s, &ws)) != SW_OK) {
            ctx_pinned_release(ctx);
            return rc;
        }
        TbPair *d_fast = static_cast<TbPair *>(ws);
        uint64_t *d_choice = reinterpret_cast<uint64_t *>(static_cast<unsigned char *>(ws) + pair_bytes);
        if ((rc = ctx_pinned_commit(ctx, d_fast, rec_bytes, s)) != SW_OK) {
            cudaFreeAsync(ws, s);
            return rc;
        }
        e = launch_tb_fill(d_fast, (int32_t)n_fast, d_choice, ranges, n_ranges, blocks, q_seqs,
                           r_seqs, out_ops, out_n_ops, score_matrix, alphabet_size, gap_open,
                           gap_extend, s);
        cudaFreeAsync(ws, s);  // stream-ordered: after the kernels that use it
        if (e != cudaSuccess)
            return set_error(SW_ECUDA, (std::string("sw_traceback: ") + cudaGetErrorString(e)).c_str());
    }

    // ---- general path: one CTA per pair, chunks whose choice bytes fit the budget
    return run_general(ctx, pairs, q_seqs, r_seqs, out_ops, out_n_ops, score_matrix, alphabet_size,
                       gap_open, gap_extend, s, "sw_traceback");
}


extern "C" int sw_cigar_capacity_device(const int32_t *results, int32_t n_pairs, int64_t *offsets,
                                        void *stream) {
    if (n_pairs < 0 || !offsets || (n_pairs > 0 && !results))
        return set_error(SW_EINVAL, "sw_cigar_capacity_device: bad argument");
    cigar_capacity_kernel<<<1, kCapThreads, 0, (cudaStream_t)stream>>>(results, n_pairs, offsets);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(SW_ECUDA, (std::string("sw_cigar_capacity_device: ") + cudaGetErrorString(e)).c_str());
    return SW_OK;
}

extern "C" int sw_traceback_device(sw_ctx *ctx, const uint8_t *q_seqs, const int64_t *q_offsets,
                                   const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                                   const int8_t *score_matrix, int32_t alphabet_size,
                                   int32_t gap_open, int32_t gap_extend, const int32_t *results,
                                   const int64_t *cigar_offsets, uint32_t *out_ops,
                                   int32_t *out_n_ops, void *stream) {
    const char *who = "sw_traceback_device";
    if (!ctx) return set_error(SW_EINVAL, "sw_traceback_device: ctx is NULL");
    if (n_pairs < 0 || (n_pairs > 0 && (!q_offsets || !r_offsets || !results || !cigar_offsets ||
                                        !out_n_ops || !q_seqs || !r_seqs || !out_ops)))
        return set_error(SW_EINVAL, "sw_traceback_device: bad argument");
    if (n_pairs == 0) return SW_OK;
    std::string msg;
    int rc = check_batch(nullptr, nullptr, 0, score_matrix, alphabet_size, gap_open, gap_extend,
                         nullptr, nullptr, nullptr, &msg);
    if (rc != SW_OK) return set_error(rc, ("sw_traceback_device: " + msg).c_str());
    int smax = 0;
    bool bytes_ok = true;
    for (int k = 0; k < alphabet_size * alphabet_size; ++k) {
        smax = std::max(smax, std::abs((int)score_matrix[k]));
        const int v = (int)score_matrix[k] - gap_open;
        bytes_ok = bytes_ok && v >= -128 && v <= 127;
    }
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    const int dev = ctx_device(ctx);
    if (dev != dev_prev && cudaSetDevice(dev) != cudaSuccess)
        return set_error(SW_ECUDA, "sw_traceback_device: cudaSetDevice failed");
    struct Restore {
        int dev, prev;
        ~Restore() {
            if (dev != prev && prev >= 0) cudaSetDevice(prev);
        }
    } restore{dev, dev_prev};
    cudaStream_t s = (cudaStream_t)stream;
    {
        // the call reads a summary back and waits for it: not capturable
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess)
            return set_error(SW_ECUDA, "sw_traceback_device: cudaStreamIsCapturing failed");
        if (cs != cudaStreamCaptureStatusNone)
            return set_error(SW_EINVAL, "sw_traceback_device: the stream is being captured (the "
                                        "call waits for its classification kernels)");
    }
    const int64_t n = n_pairs;
    cudaError_t e = cudaMemsetAsync(out_n_ops, 0, (size_t)n * sizeof(int32_t), s);
    if (e != cudaSuccess) return set_error(SW_ECUDA, "sw_traceback_device: memset failed");

    // planning workspace: summary | slot counts | slot words | slot cursors
    // (records, words) | fast-path records | general-path records
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_count = up(sizeof(TbDevSummary));
    const size_t o_words = o_count + up((size_t)kTbSlots * 4);
    const size_t o_pos = o_words + up((size_t)kTbSlots * 8);
    const size_t o_wpos = o_pos + up((size_t)kTbSlots * 4);
    const size_t o_rec = o_wpos + up((size_t)kTbSlots * 8);
    const size_t o_gen = o_rec + up((size_t)n * sizeof(TbPair));
    const size_t ws_bytes = o_gen + up((size_t)n * sizeof(CigarPair));
    void *ws = nullptr;
    if ((rc = ctx_alloc_async(ctx, ws_bytes, s, &ws)) != SW_OK) return rc;
    unsigned char *wb = static_cast<unsigned char *>(ws);
    TbDevArgs a;
    a.qo = q_offsets;
    a.ro = r_offsets;
    a.co = cigar_offsets;
    a.res = results;
    a.n = n;
    a.unit = (int64_t)-gap_open - gap_extend + smax;
    a.bytes_ok = bytes_ok ? 1 : 0;
    a.sum = reinterpret_cast<TbDevSummary *>(wb);
    a.slot_count = reinterpret_cast<uint32_t *>(wb + o_count);
    a.slot_words = reinterpret_cast<unsigned long long *>(wb + o_words);
    a.slot_pos = reinterpret_cast<uint32_t *>(wb + o_pos);
    a.slot_wpos = reinterpret_cast<unsigned long long *>(wb + o_wpos);
    a.records = reinterpret_cast<TbPair *>(wb + o_rec);
    a.general = reinterpret_cast<CigarPair *>(wb + o_gen);
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    e = cudaMemsetAsync(wb, 0, o_pos, s);  // summary, slot counts and words
    if (e == cudaSuccess) {
        tb_dev_classify<<<grid, 256, 0, s>>>(a);
        tb_dev_scan<<<1, kTbScanThreads, 0, s>>>(a);
        tb_dev_scatter<<<grid, 256, 0, s>>>(a);
        e = cudaGetLastError();
    }
    TbDevSummary hs;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, a.sum, sizeof hs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFreeAsync(ws, s);
        return set_error(SW_ECUDA, (std::string("sw_traceback_device: ") + cudaGetErrorString(e)).c_str());
    }
    if (hs.err != 0) {
        cudaFreeAsync(ws, s);
        const unsigned long long code = ~hs.err;
        const long long p = (long long)(code >> 3);
        const int kind = (int)(code & 7);
        char buf[160];
        if (kind == 3)
            snprintf(buf, sizeof buf, "%s: offsets of pair %lld negative or decreasing", who, p);
        else if (kind == 4)
            snprintf(buf, sizeof buf, "%s: pair %lld has a length above SW_MAX_LEN", who, p);
        else if (kind == 1)
            snprintf(buf, sizeof buf, "%s: pair %lld has coordinates outside it", who, p);
        else
            snprintf(buf, sizeof buf, "%s: pair %lld needs more ops of room than its cigar offsets give",
                     who, p);
        return set_error(SW_ERANGE, buf);
    }
    if (hs.n_fast > 0) {
        void *cw = nullptr;
        if ((rc = ctx_alloc_async(ctx, (size_t)hs.words * 8, s, &cw)) != SW_OK) {
            cudaFreeAsync(ws, s);
            return rc;
        }
        e = launch_tb_fill(a.records, hs.n_fast, static_cast<uint64_t *>(cw), hs.ranges,
                           hs.n_ranges, hs.blocks, q_seqs, r_seqs, out_ops, out_n_ops, score_matrix,
                           alphabet_size, gap_open, gap_extend, s);
        cudaFreeAsync(cw, s);  // stream-ordered: after the kernel that uses it
        if (e != cudaSuccess) {
            cudaFreeAsync(ws, s);
            return set_error(SW_ECUDA, (std::string("sw_traceback_device: ") + cudaGetErrorString(e)).c_str());
        }
    }
    std::vector<CigarPair> pairs;
    if (hs.n_general > 0) {
        pairs.resize((size_t)hs.n_general);
        e = cudaMemcpyAsync(pairs.data(), a.general, pairs.size() * sizeof(CigarPair),
                            cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFreeAsync(ws, s);
            return set_error(SW_ECUDA, (std::string("sw_traceback_device: ") + cudaGetErrorString(e)).c_str());
        }
        // in pair order, as the host preparation lists them
        std::sort(pairs.begin(), pairs.end(),
                  [](const CigarPair &x, const CigarPair &y) { return x.id < y.id; });
    }
    cudaFreeAsync(ws, s);  // stream-ordered: after the fill kernel reads the records
    return run_general(ctx, pairs, q_seqs, r_seqs, out_ops, out_n_ops, score_matrix, alphabet_size,
                       gap_open, gap_extend, s, who);
}
