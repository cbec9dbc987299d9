// Device side of graph preparation (sm_103a): adjacency bitmaps of the
// highest-ranked vertices, built from the CSR already in device memory.
//
// Bitmap i (words 32-bit words, bit c set when c is a neighbour) belongs to
// internal vertex n-1-i, i < nh; hub[r] is that index for the nh top ranks
// and -1 for every other vertex.  Every column id lies in [0, n) (the host
// relabelled validated ids), so each bit lands inside its own bitmap.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "internal.hpp"

namespace pm {
namespace {

__global__ void hub_index_kernel(int64_t n, int64_t nh, int32_t *__restrict__ hub) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride)
        hub[r] = r >= n - nh ? int32_t(n - 1 - r) : -1;
}

// One block per hub row at a time; the row's ids are read coalesced and
// OR-ed into the bitmap (a bitmap of n bits is shared by the block's threads).
__global__ void hub_bits_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                int64_t n, int64_t nh, int64_t words, uint32_t *__restrict__ bits) {
    for (int64_t i = blockIdx.x; i < nh; i += gridDim.x) {
        const int64_t r = n - 1 - i;
        uint32_t *w = bits + i * words;
        const int64_t end = rowptr[r + 1];
        for (int64_t e = rowptr[r] + threadIdx.x; e < end; e += blockDim.x) {
            const uint32_t c = uint32_t(col[e]);
            atomicOr(w + (c >> 5), 1u << (c & 31u));
        }
    }
}

}  // namespace

int launch_hub_bitmaps(const int64_t *d_rowptr, const int32_t *d_col, int64_t n, int64_t nh,
                       int64_t words, int32_t *d_hub, uint32_t *d_bits, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_bits, 0, sizeof(uint32_t) * size_t(nh) * size_t(words), s);
    if (e != cudaSuccess) return int(e);
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t idx_blocks = std::min<int64_t>((n + 255) / 256, int64_t(sms) * 8);
    hub_index_kernel<<<unsigned(idx_blocks), 256, 0, s>>>(n, nh, d_hub);
    const int64_t bit_blocks = std::min<int64_t>(nh, int64_t(sms) * 8);
    hub_bits_kernel<<<unsigned(bit_blocks), 256, 0, s>>>(d_rowptr, d_col, n, nh, words, d_bits);
    return int(cudaGetLastError());
}

}  // namespace pm
