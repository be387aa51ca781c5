// lbm_conserved_noalloc: the conserved totals of lbm_conserved() computed without allocating any
// device memory during the call.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they want the totals --
// for instance code running inside a host framework that owns all device memory through its own
// pool and forbids raw allocations, code that must not trigger the device-wide synchronisation an
// allocation can cause (a latency-sensitive monitoring loop beside other GPU work), or a caller
// that has already reserved every byte it is allowed.  The regular entry point uses a per-context
// scratch array allocated when the grid is built; this one uses a fixed-size array that lives in
// the library's device code instead.
//
// The per-block partial sums go to `g_ledger_scratch`, a file-scope device array of
// kLedgerMaxBlocks x 5 doubles (20 MiB), held by every GPU on which the library's device code is
// loaded, until the process exits.  Host code cannot use the array's name as a device address; the
// address is looked up with cudaGetSymbolAddress the first time a call runs on a device (so that
// first call should come before any stream capture) and passed to the kernels.  The address is
// cached per device together with the driver context it belongs to: if the device's context was
// torn down and recreated (cudaDeviceReset by the host framework), the next call looks it up
// again instead of using an address of the old context.
// The totals stay on the device, so this call cannot report non-finite values the way
// lbm_conserved does (LBM_ERR_NONFINITE): a caller that needs that check reads d_out after
// lbm_sync() and tests it.
// Every call shares the array and it keeps the last call's contents: each call overwrites the
// partials it reads before reading them, so nothing has to be cleared, but two calls whose work
// overlaps on the GPU (different streams, different contexts on one device) race on the array.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbmtree.h"
#include "kernels.h"

namespace lbm {
int ledger_launch_args(lbm_ctx* c, StepArgs* a, long long* nblocks, KernelSet* ks, cudaStream_t* s, int* device);
int set_error(int code, const std::string& msg);
}  // namespace lbm

namespace {
constexpr long long kLedgerMaxBlocks = 1ll << 19;
__device__ __align__(256) double g_ledger_scratch[kLedgerMaxBlocks * 5];

std::mutex g_mu;
double* g_addr[256] = {nullptr};
CUcontext g_ctx[256] = {nullptr};   // the driver context g_addr[d] was looked up in

// The calling thread's current driver context (nullptr if it cannot be queried).  The driver
// entry point is fetched through the runtime, so the library needs no link to libcuda.
CUcontext current_context() {
    using GetCurrent = CUresult (*)(CUcontext*);
    static GetCurrent fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<GetCurrent>(p);
    }();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}
}  // namespace

extern "C" int lbm_conserved_noalloc(lbm_ctx* ctx, double* d_out) {
    using namespace lbm;
    if (!ctx || !d_out) return set_error(LBM_ERR_ARG, "null context or output pointer");
    StepArgs a;
    long long nb = 0;
    KernelSet ks;
    cudaStream_t stream = nullptr;
    int device = 0;
    if (int r = ledger_launch_args(ctx, &a, &nb, &ks, &stream, &device)) return r;
    if (nb > kLedgerMaxBlocks)
        return set_error(LBM_ERR_ARG, "grid has " + std::to_string(nb) + " blocks; lbm_conserved_noalloc supports at most " +
                                          std::to_string(kLedgerMaxBlocks) + " (use lbm_conserved)");
    if (device < 0 || device >= 256) return set_error(LBM_ERR_ARG, "device index out of range");
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        // the context's device is current here (ledger_launch_args sets it)
        const CUcontext cur = current_context();
        if (!g_addr[device] || !cur || cur != g_ctx[device]) {
            g_ctx[device] = cur;
            cudaError_t e = cudaGetSymbolAddress((void**)&g_addr[device], g_ledger_scratch);
            if (e != cudaSuccess) {
                g_addr[device] = nullptr;
                return set_error(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        scratch = g_addr[device];
    }
    ks.ledger(a, nb, scratch, d_out, stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("ledger launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}
