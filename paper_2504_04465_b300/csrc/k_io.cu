// Host-order <-> slot-order transfer of per-cell fields on the device.  The library lists cells
// level by level (lbm_cells order); on the device every level stores them in block slots.  A
// per-level table slot[k] (k: listing index within the level) moves fields between the two
// layouts, so that initialisation and readout copy one contiguous array per field.
#include <cuda_runtime.h>

namespace lbm {

namespace {

__global__ void k_scatter(const int* __restrict__ slot, long long count, const double* __restrict__ src,
                          long long src_stride, int ncomp, double* __restrict__ dst, long long dst_stride) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const long long s = slot[i];
    for (int c = 0; c < ncomp; ++c) dst[c * dst_stride + s] = src[c * src_stride + i];
}

__global__ void k_gather(const int* __restrict__ slot, long long count, const double* __restrict__ src,
                         long long src_stride, int ncomp, double* __restrict__ dst, long long dst_stride) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const long long s = slot[i];
    for (int c = 0; c < ncomp; ++c) dst[c * dst_stride + i] = src[c * src_stride + s];
}

}  // namespace

// dst[c][slot[i]] = src[c][i], i < count
void launch_scatter(const int* slot, long long count, const double* src, long long src_stride, int ncomp, double* dst,
                    long long dst_stride, cudaStream_t s) {
    if (count) k_scatter<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(slot, count, src, src_stride, ncomp, dst, dst_stride);
}

// dst[c][i] = src[c][slot[i]], i < count
void launch_gather(const int* slot, long long count, const double* src, long long src_stride, int ncomp, double* dst,
                   long long dst_stride, cudaStream_t s) {
    if (count) k_gather<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(slot, count, src, src_stride, ncomp, dst, dst_stride);
}

}  // namespace lbm
