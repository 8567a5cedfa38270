// 2-bit packed DNA input.  Residue k of a packed stream sits in byte k >> 2,
// bits 2 (k & 3) .. 2 (k & 3) + 1 (four residues per byte, the first in the
// low bits).  Packed input moves a quarter of the bytes host to device and
// through the serving staging; on the device the stream is expanded once
// per execution into one byte per residue, the form the alignment kernels
// read.  The expansion moves about 1.25 bytes per residue through HBM, a few
// microseconds for the 100k-pair DNA batch against milliseconds of
// integer-bound alignment, so the kernels need no packed variant.
#include <cuda_runtime.h>

#include <algorithm>

#include "sw_internal.h"
#include "swgb.h"

namespace swgb {
namespace {

// Thread per packed byte, four residues out as one 32-bit store.
__global__ void unpack_2bit_kernel(const uint8_t *__restrict__ packed, int64_t n_res,
                                   uint8_t *__restrict__ out) {
    const int64_t n_full = n_res >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_full; b += stride) {
        const uint32_t v = packed[b];
        const uint32_t w = (v & 3u) | (((v >> 2) & 3u) << 8) | (((v >> 4) & 3u) << 16) |
                           ((v >> 6) << 24);
        reinterpret_cast<uint32_t *>(out)[b] = w;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int64_t k = n_full << 2; k < n_res; ++k)
            out[k] = (uint8_t)((packed[k >> 2] >> (2 * (k & 3))) & 3u);
    }
}

}  // namespace

cudaError_t enqueue_unpack_2bit(const uint8_t *packed, int64_t n_res, uint8_t *out, int sms,
                                cudaStream_t s) {
    if (n_res <= 0) return cudaSuccess;
    const int64_t bytes = (n_res + 3) >> 2;
    const int threads = 256;
    const int64_t want = (bytes + threads - 1) / threads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    unpack_2bit_kernel<<<grid, threads, 0, s>>>(packed, n_res, out);
    return cudaGetLastError();
}

}  // namespace swgb

using namespace swgb;

extern "C" int sw_pack_2bit(const uint8_t *codes, int64_t n_res, uint8_t *packed) {
    if (n_res < 0 || (n_res > 0 && (!codes || !packed)))
        return set_error(SW_EINVAL, "sw_pack_2bit: bad argument");
    for (int64_t b = 0; b < (n_res + 3) >> 2; ++b) {
        uint8_t v = 0;
        for (int k = 0; k < 4; ++k) {
            const int64_t i = 4 * b + k;
            if (i >= n_res) break;
            if (codes[i] > 3) return set_error(SW_ERANGE, "sw_pack_2bit: code above 3");
            v |= (uint8_t)(codes[i] << (2 * k));
        }
        packed[b] = v;
    }
    return SW_OK;
}

extern "C" int sw_unpack_2bit(const uint8_t *packed, int64_t n_res, uint8_t *codes,
                              void *stream) {
    if (n_res < 0 || (n_res > 0 && (!packed || !codes)))
        return set_error(SW_EINVAL, "sw_unpack_2bit: bad argument");
    if ((reinterpret_cast<uintptr_t>(codes) & 3u) != 0)
        return set_error(SW_EINVAL, "sw_unpack_2bit: codes must be 4-byte aligned");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const cudaError_t e = enqueue_unpack_2bit(packed, n_res, codes, std::max(sms, 1),
                                              (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(SW_ECUDA, "sw_unpack_2bit: launch failed");
    return SW_OK;
}
