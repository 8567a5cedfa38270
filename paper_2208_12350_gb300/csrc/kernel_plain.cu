// One thread block per pair: the plain launch form, and the general int32
// path for pairs whose scores exceed the batched kernel's scaled range.
//
// ADEPT's parallelisation (Section II-B.2, Fig. 3): the cells of one
// anti-diagonal are computed at once, each thread owning one strip of the
// matrix and waiting one step per position for its neighbour.  Here thread
// t owns query rows [t*k, t*k + k) (k = 1 unless n > blockDim.x) and works
// on column j = step - t.  Neighbour values go through shared memory on a
// path every thread takes: each step every thread writes its last row's H
// and F and reads its upper neighbour's, one barrier per step.  That is the
// exchange GEVO's edits 5, 6, 8 and 10 converged on (Section VI-A): the
// register shuffle with a shared-memory special case for warp edges
// diverged inside every warp and cost more than it saved.  The boundary is
// initialised once (Section VI-C: a per-thread re-initialisation of shared
// memory with barriers was ADEPT-V0's bottleneck).
//
// Scores are plain int32.  The maximal cell is tracked per thread as
// (H, j, i) under the end rule and reduced over the block; the reverse pass
// (Fig. 2(c)) reruns the sweep on the reversed prefixes.
#include "sw_internal.h"

namespace swgb {
namespace {

__device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }

__device__ __forceinline__ uint64_t block_max_u64(uint64_t v, uint64_t *red) {
    for (int off = 16; off > 0; off >>= 1) {
        uint64_t o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o > v ? o : v;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red[lane] : 0;
        for (int off = 16; off > 0; off >>= 1) {
            uint64_t o = __shfl_xor_sync(0xffffffffu, v, off);
            v = o > v ? o : v;
        }
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    v = red[0];
    __syncthreads();
    return v;
}

// Key of a cell under the end rule: larger H, then smaller j, then smaller i.
__device__ __forceinline__ uint64_t cell_key(int h, int j, int i) {
    return h > 0 ? ((uint64_t)(uint32_t)h << 32) | ((uint64_t)(0xFFFF - j) << 16) |
                       (uint64_t)(0xFFFF - i)
                 : 0ull;
}

// Local-alignment sweep over a (n rows, read at a[i * a_step]) against
// b (m columns, read at b[j * b_step]).  Returns the block-wide best key.
template <int KMAX>
__device__ uint64_t plain_sweep(const uint8_t *a, int a_step, int n, const uint8_t *b,
                                int b_step, int m, const int *smat, int A, int go, int ge,
                                int *xH, int *xF, uint64_t *red) {
    const int T = blockDim.x, t = threadIdx.x;
    if (n <= 0 || m <= 0) return 0ull;
    const int k = (n + T - 1) / T;  // rows per thread, <= KMAX (host checks)
    const int nthr = (n + k - 1) / k;
    const int row0 = t * k;
    const int rows = max(0, min(k, n - row0));
    // KMAX == 1 keeps the row in registers; the many-rows variant keeps its
    // rows in thread-local memory (long queries only).
    int Hl[KMAX], E[KMAX], qa[KMAX];
    const int row_loop = KMAX == 1 ? 1 : rows;  // compile-time 1 keeps registers
#pragma unroll
    for (int r = 0; r < row_loop; ++r) {
        if (r >= rows) break;
        Hl[r] = 0;
        E[r] = kPlainNegInf;
        qa[r] = min((int)a[(ptrdiff_t)(row0 + r) * a_step], A - 1) * A;
    }
    for (int idx = t; idx < 2 * T; idx += T) {
        xH[idx] = 0;
        xF[idx] = kPlainNegInf;
    }
    __syncthreads();
    int bestH = 0, bestJ = 0, bestI = 0;
    int prev_up = 0;  // H of the row above at the previous column
    const int steps = m + nthr - 1;
    for (int s = 0; s < steps; ++s) {
        const int j = s - t;
        const int rb = ((s + 1) & 1) * T;  // buffer written at step s - 1
        int upH = 0, upF = kPlainNegInf;
        if (t > 0) {
            upH = xH[rb + t - 1];
            upF = xF[rb + t - 1];
        }
        int myH = 0, myF = kPlainNegInf;
        if (rows > 0 && j >= 0 && j < m) {
            const int bc = min((int)b[(ptrdiff_t)j * b_step], A - 1);
            int diag = prev_up;
            int F = imax(upF + ge, upH + go);
            int h = 0;
#pragma unroll
            for (int r = 0; r < row_loop; ++r) {
                if (r >= rows) break;
                if (r > 0) F = imax(F + ge, h + go);
                const int hl = Hl[r];
                E[r] = imax(E[r] + ge, hl + go);
                int v = imax(diag + smat[qa[r] + bc], E[r]);
                v = imax(imax(v, F), 0);
                diag = hl;
                Hl[r] = v;
                h = v;
                if (v > bestH) {  // first (j, i) in visiting order keeps ties
                    bestH = v;
                    bestJ = j;
                    bestI = row0 + r;
                }
            }
            myH = h;
            myF = F;
        }
        prev_up = upH;
        const int wb = (s & 1) * T;
        xH[wb + t] = myH;
        xF[wb + t] = myF;
        __syncthreads();
    }
    return block_max_u64(cell_key(bestH, bestJ, bestI), red);
}

template <int KMAX>
__device__ __forceinline__ void plain_pair(const PlainParams &p, const PairInfo &pi,
                                           const int *smat, int *xH, int *xF, uint64_t *red);

template <int KMAX>
__global__ void __launch_bounds__(KMAX == 1 ? 1024 : kPlainWideThreads)
    sw_plain_kernel(const __grid_constant__ PlainParams p) {
    extern __shared__ __align__(16) int smem_plain[];
    const int A = p.alphabet;
    const int T = blockDim.x;
    const int mat_words = (A * A + 3) & ~3;
    int *smat = smem_plain;
    int *xH = smat + mat_words;
    int *xF = xH + 2 * T;
    uint64_t *red = reinterpret_cast<uint64_t *>(xF + 2 * T);
    for (int i = threadIdx.x; i < A * A; i += T) smat[i] = p.mat[i];
    __syncthreads();

    int first = 0, count = p.n_pairs;
    if (p.range) {
        first = p.range[0];
        count = p.range[1];
    }
    // block-uniform loop: every barrier inside is reached by the whole block
    for (int b = blockIdx.x; b < count; b += gridDim.x)
        plain_pair<KMAX>(p, p.pairs[first + b], smat, xH, xF, red);
}

template <int KMAX>
__device__ __forceinline__ void plain_pair(const PlainParams &p, const PairInfo &pi,
                                           const int *smat, int *xH, int *xF, uint64_t *red) {
    const int A = p.alphabet;
    const uint8_t *q = p.q + pi.q;
    const uint8_t *r = p.r + pi.r;
    const uint64_t key = plain_sweep<KMAX>(q, 1, pi.n, r, 1, pi.m, smat, A, p.gap_open,
                                           p.gap_extend, xH, xF, red);
    const int S = (int)(key >> 32);
    int o0 = 0, o1 = -1, o2 = -1, o3 = -1, o4 = -1;
    if (S > 0 && p.ends_only) {
        o0 = S;
        o1 = 0xFFFF - (int)(key & 0xFFFF);
        o2 = 0xFFFF - (int)((key >> 16) & 0xFFFF);
    } else if (S > 0) {  // block-uniform
        const int rend = 0xFFFF - (int)((key >> 16) & 0xFFFF);
        const int qend = 0xFFFF - (int)(key & 0xFFFF);
        const uint64_t k2 = plain_sweep<KMAX>(q + qend, -1, qend + 1, r + rend, -1, rend + 1,
                                              smat, A, p.gap_open, p.gap_extend, xH, xF, red);
        const int S2 = (int)(k2 >> 32);
        const int l = 0xFFFF - (int)((k2 >> 16) & 0xFFFF);
        const int kk = 0xFFFF - (int)(k2 & 0xFFFF);
        if (S2 != S && threadIdx.x == 0) atomicOr(p.status, kStatusReverseMismatch);
        o0 = S;
        o1 = qend;
        o2 = rend;
        o3 = qend - kk;
        o4 = rend - l;
    }
    if (threadIdx.x == 0) {
        p.out.score[pi.id] = o0;
        p.out.qend[pi.id] = o1;
        p.out.rend[pi.id] = o2;
        if (!p.ends_only) {
            p.out.qstart[pi.id] = o3;
            p.out.rstart[pi.id] = o4;
        }
    }
}

__global__ void check_residues_kernel(const uint8_t *s, int64_t n, int A,
                                      unsigned long long *bad) {
    unsigned long long local = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        local += s[i] >= A;
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(bad, local);
}

__global__ void guard_fill_kernel(const GuardList g) {
    for (int r = blockIdx.y; r < g.n; r += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.words[r];
             i += gridDim.x * blockDim.x)
            g.ptr[r][i] = kGuardWord;
}

__global__ void guard_check_kernel(const GuardList g, int32_t *status) {
    bool bad = false;
    for (int r = blockIdx.y; r < g.n; r += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.words[r];
             i += gridDim.x * blockDim.x)
            bad |= g.ptr[r][i] != kGuardWord;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusGuard);
}

}  // namespace

cudaError_t launch_guard_fill(const GuardList &g, cudaStream_t s) {
    if (g.n <= 0) return cudaSuccess;
    guard_fill_kernel<<<dim3(4, g.n), 256, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_guard_check(const GuardList &g, int32_t *status, cudaStream_t s) {
    if (g.n <= 0) return cudaSuccess;
    guard_check_kernel<<<dim3(4, g.n), 256, 0, s>>>(g, status);
    return cudaGetLastError();
}

size_t plain_smem_bytes(int threads, int alphabet) {
    const int mat_words = (alphabet * alphabet + 3) & ~3;
    return (size_t)(mat_words + 4 * threads) * sizeof(int) + 32 * sizeof(uint64_t);
}

cudaError_t launch_plain(const PlainParams &p, int threads, int rows_per_thread_max,
                         cudaStream_t s) {
    if (p.n_pairs <= 0) return cudaSuccess;
    const size_t smem = plain_smem_bytes(threads, p.alphabet);
    // at most 4 KB of matrix + 16 KB of exchange buffers: under the 48 KB default
    if (rows_per_thread_max <= 1)
        sw_plain_kernel<1><<<p.n_pairs, threads, smem, s>>>(p);
    else
        sw_plain_kernel<kPlainMaxRows><<<p.n_pairs, kPlainWideThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_plain_range(const PlainParams &p, int threads, int rows_per_thread_max,
                               int grid, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    if (rows_per_thread_max <= 1) {
        sw_plain_kernel<1><<<grid, threads, plain_smem_bytes(threads, p.alphabet), s>>>(p);
    } else {
        sw_plain_kernel<kPlainMaxRows>
            <<<grid, kPlainWideThreads, plain_smem_bytes(kPlainWideThreads, p.alphabet), s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_check_residues(const uint8_t *seqs, int64_t n, int alphabet,
                                  unsigned long long *bad, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n <= 0) return e;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    check_residues_kernel<<<(int)blocks, 256, 0, s>>>(seqs, n, alphabet, bad);
    return cudaGetLastError();
}

}  // namespace swgb
