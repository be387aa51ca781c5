// Host-order <-> slot-order transfer of per-cell fields on the device.  The library lists cells
// level by level (lbm_cells order); on the device every level stores them in block slots.  A
// per-level table slot[k] (k: listing index within the level) moves fields between the two
// layouts, so that initialisation and readout copy one contiguous array per field.
#include <cuda_runtime.h>

#include "kernels.h"

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

// Remesh transfer: dst[c][r] = sum_k w[k] src_level(col[k])[c][slot(col[k])] over the row's
// entries k in [rowptr[r], rowptr[r + 1]); col packs (old level << 40) | old slot.
__global__ void k_transfer(const long long* __restrict__ rowptr, const long long* __restrict__ col,
                           const double* __restrict__ w, long long rows, TransferSrc src, int ncomp,
                           double* __restrict__ dst) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const long long k0 = rowptr[r], k1 = rowptr[r + 1];
    for (int c = 0; c < ncomp; ++c) {
        double acc = 0.0;
        for (long long k = k0; k < k1; ++k) {
            const int lev = (int)(col[k] >> 40);
            const long long slot = col[k] & ((1ll << 40) - 1);
            acc += w[k] * src.ptr[lev][(long long)c * src.ncell[lev] + slot];
        }
        dst[(long long)c * rows + r] = acc;
    }
}

}  // namespace

void launch_transfer(const long long* rowptr, const long long* col, const double* w, long long rows,
                     const TransferSrc& src, int ncomp, double* dst, cudaStream_t s) {
    if (rows) k_transfer<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(rowptr, col, w, rows, src, ncomp, dst);
}

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
