// Device-side storage formats and the block-table gather of the CUDA path.
//
// Layout (Sec. 4.4 of arXiv 2504.04465, adapted to blocks): every level stores its cells in
// fixed-size blocks (BX x BY x BZ, x fastest), blocks in Morton order; populations are SoA inside
// a block, f[(block * Q + q) * BS + local] (cell = block * BS + local), so one block's Q arrays
// are contiguous and population q of a gathered cell is an immediate offset q * BS.  Two buffers per level (A/B, the
// "two-population" storage of Sec. 4.1).  The stored state of a cell is its post-collision
// populations; a step gathers f_i(x) = f*_i(x - xi_i) from the other buffer (pull form of
// Eqs. CollisionStep/StreamingStep), collides and writes its own slot.  The weakly compressible
// models store and compute deviations f_i - w_i rho_ref (FP64/FP32 plain, binary16 relative), so
// that FP32 rounding acts on small numbers.
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

#include "device_types.h"
#include "lattice_tables.h"

namespace lbm {

template <int ST> struct Store;

template <> struct Store<ST_F64> {
    using T = double;     // arithmetic type
    using S = double;     // stored type
    template <bool DEV> static __device__ __forceinline__ T load(const void* p, long long i, T) { return __ldg((const double*)p + i); }
    template <bool DEV> static __device__ __forceinline__ void store(void* p, long long i, T v, T) { ((double*)p)[i] = v; }
};

template <> struct Store<ST_F32> {
    using T = float;
    using S = float;
    template <bool DEV> static __device__ __forceinline__ T load(const void* p, long long i, T) { return __ldg((const float*)p + i); }
    template <bool DEV> static __device__ __forceinline__ void store(void* p, long long i, T v, T) { ((float*)p)[i] = v; }
};

// binary16 deviation relative to the reference value ref = w_i rho_ref (or the g reference):
// stored d = v / ref - 1, computed as v * (1 / ref) (round to nearest even); arithmetic in FP32.
// With DEV the arithmetic value is itself the deviation v - ref (weakly compressible models),
// else the population v.  load() takes ref, store() takes 1 / ref.
template <> struct Store<ST_F16DEV> {
    using T = float;
    using S = __half;
    template <bool DEV> static __device__ __forceinline__ T load(const void* p, long long i, T ref) {
        const float h = __half2float(__ldg((const __half*)p + i));
        return DEV ? ref * h : ref * (1.0f + h);
    }
    template <bool DEV> static __device__ __forceinline__ void store(void* p, long long i, T v, T inv_ref) {
        ((__half*)p)[i] = __float2half_rn(DEV ? v * inv_ref : fmaf(v, inv_ref, -1.0f));
    }
};

// storage index of population q of cell (= block * BS + local)
template <int BS, int Q>
__device__ __forceinline__ long long pidx(long long cell, int q) {
    const long long b = cell / BS;
    return (b * Q + q) * BS + (cell - b * BS);
}

__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// source cell of the pull for velocity (cx, cy, cz) from local (lx, ly, lz) of block b
template <int BX, int BY, int BZ>
__device__ __forceinline__ long long src_cell(const int* nbr_s, long long b, int lx, int ly, int lz,
                                              int cx, int cy, int cz) {
    int sx = lx - cx, sy = ly - cy, sz = lz - cz;
    const int ox = sx < 0 ? -1 : (sx >= BX ? 1 : 0);
    const int oy = sy < 0 ? -1 : (sy >= BY ? 1 : 0);
    const int oz = sz < 0 ? -1 : (sz >= BZ ? 1 : 0);
    sx -= ox * BX; sy -= oy * BY; sz -= oz * BZ;
    const int k = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
    const long long nb = (k == 13) ? b : (long long)nbr_s[k];
    if (nb < 0) return -1;
    return nb * (BX * BY * BZ) + (sz * BY + sy) * BX + sx;
}

// same through the level's global neighbour table (cells of another block / level)
template <int BX, int BY, int BZ>
__device__ __forceinline__ long long src_cell_g(const int* nbr, long long cell, int cx, int cy, int cz) {
    constexpr int BS = BX * BY * BZ;
    const long long b = cell / BS;
    const int l = int(cell - b * BS);
    const int lx = l % BX, ly = (l / BX) % BY, lz = l / (BX * BY);
    int sx = lx - cx, sy = ly - cy, sz = lz - cz;
    const int ox = sx < 0 ? -1 : (sx >= BX ? 1 : 0);
    const int oy = sy < 0 ? -1 : (sy >= BY ? 1 : 0);
    const int oz = sz < 0 ? -1 : (sz >= BZ ? 1 : 0);
    sx -= ox * BX; sy -= oy * BY; sz -= oz * BZ;
    const int k = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
    const long long nb = (k == 13) ? b : (long long)__ldg(nbr + b * 27 + k);
    if (nb < 0) return -1;
    return nb * BS + (sz * BY + sy) * BX + sx;
}

}  // namespace lbm
