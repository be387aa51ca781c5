// Host-visible entry points of the kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include "device_types.h"
#include "../../include/lbmtree.h"

namespace lbm {

constexpr int MAX_VARIANTS = 8;     // lbm_variants() fills at most this many codes

struct KernelSet {
    // interior-kernel launch on s_fast, general-kernel launch on s_gen (they touch disjoint cells
    // and may run concurrently)
    void (*step)(const StepArgs&, long long n_fast, long long n_gen, cudaStream_t s_fast, cudaStream_t s_gen) = nullptr;
    // which: 0 moments, 1 f, 2 g, 3 lambda, 4..6 the same three with coarse-ghost unknowns
    // coalesced (the conserved state; f as stored: deviations in the deviation formats), 7 the
    // kinetic sensor eps
    void (*read)(const StepArgs&, int lev, int which, double* out, cudaStream_t) = nullptr;
    // pre-collision state as stored (f, g, lambda; slot-indexed) into a level's buffers
    void (*load_state)(const StepArgs&, int lev, const double* full, cudaStream_t) = nullptr;
    // after a remesh: concave-corner coarse ghosts of level lev reproduce their carried state
    void (*remesh_corners)(const StepArgs&, int lev, cudaStream_t) = nullptr;
    void (*ledger)(const StepArgs&, long long nblocks, double* partial, double* out, cudaStream_t) = nullptr;
    void (*init)(const StepArgs&, int lev, const double* rho, const double* u, const double* T, cudaStream_t) = nullptr;
    // AA-pattern streaming (one buffer, single level): one iteration of parity a.rd[0]; null
    // where the model is not compiled with it
    void (*aa)(const StepArgs&, cudaStream_t) = nullptr;
    const void* step_kernel = nullptr;
    int block_threads = 0;
    // compiled variants of the step launch (occupancy targets of the simple-block kernel; codes
    // >= 100: the same target with the simple blocks gathered directly instead of staged)
    void (*variant[MAX_VARIANTS])(const StepArgs&, long long, long long, cudaStream_t, cudaStream_t) = {};
    int variant_minb[MAX_VARIANTS] = {};
    int n_variants = 1;
    // batched launches of several cases (per variant; null where the lattice has none)
    void (*batch[MAX_VARIANTS])(const StepArgs*, const long long*, const long long*, int, long long, long long,
                                cudaStream_t, cudaStream_t) = {};
};

// Kernel-set code of the recursive-regularized collision with the trace of the second-order
// moments equilibrated (public LBM_RR with trace_eq set); the other codes are the public models.
constexpr int KMODEL_RR_TRACE = 6;

// Kernels for (model, storage, block shape) of each lattice; false if that combination is not built.
bool find_kernels_d2q9(int model, int storage, const int* block, KernelSet& out);
bool find_kernels_d3q27(int model, int storage, const int* block, KernelSet& out);
bool find_kernels_d2q37(int model, int storage, const int* block, bool newton_fp32, KernelSet& out);
bool find_kernels_d2q21(int model, int storage, const int* block, bool newton_fp32, KernelSet& out);
bool find_kernels_d2q21w(int model, int storage, const int* block, KernelSet& out);
bool find_kernels_d2q13(int model, int storage, const int* block, bool newton_fp32, KernelSet& out);

int mlp_train_device(const double* d_uT, const double* d_lam, int64_t n, double T0, const lbm_mlp_train_params& p,
                     float* d_master, float* d_rounded, double* h_ms, float* h_loss, cudaStream_t s);
// per-level sources of the remesh transfer (old conserved state, slot-indexed components)
struct TransferSrc {
    const double* ptr[MAX_LEVELS];
    long long ncell[MAX_LEVELS];
};
void launch_transfer(const long long* rowptr, const long long* col, const double* w, long long rows,
                     const TransferSrc& src, int ncomp, double* dst, cudaStream_t s);
void launch_scatter(const int* slot, long long count, const double* src, long long src_stride, int ncomp, double* dst,
                    long long dst_stride, cudaStream_t s);
void launch_gather(const int* slot, long long count, const double* src, long long src_stride, int ncomp, double* dst,
                   long long dst_stride, cudaStream_t s);
void launch_newton_batch_d2q21(const double* uT, long long n, const ModelDev& m, double* lam, int* iters, cudaStream_t s);
void launch_newton_batch_d2q13(const double* uT, long long n, const ModelDev& m, double* lam, int* iters, cudaStream_t s);
void launch_newton_batch_d2q37(const double* uT, long long n, const ModelDev& m, double* lam, int* iters, cudaStream_t s);

// Constant tables of the D2Q37 and D2Q21 translation units (current device).
cudaError_t upload_tables_d2q37(const double* w37, const double* H37, double cs2_37);
cudaError_t upload_tables_d2q21(const double* w21, const double* H21);

// weights.cpp: D2Q37 weights re-derived from isotropy, Hermite tables of both lattices
void lattice_constants(double w37[37], double H37[37 * 15], double* cs2_37, double w21[21], double H21[21 * 10]);
// D2Q37 thermal-equilibrium coefficients per velocity class (FP64, and FP32 rounded to conserve
// mass, momentum and energy exactly); max_residual: largest moment error left in the FP32 table
void d2q37_class_tables(double C64[13 * 15], float C32[13 * 15], double* th64, float* th32, double* max_residual);

}  // namespace lbm
