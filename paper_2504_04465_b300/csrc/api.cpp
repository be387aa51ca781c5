// C ABI of the library (include/lbmtree.h): context, grid upload, level scheduler, CUDA graph,
// readout and the conservation ledger.
//
// Scheduler (Sec. 4.5 of arXiv 2504.04465): at fine iteration t the levels i with t % 2^i == 0
// are active; the coarsest goes first.  All active levels of an iteration run in ONE launch (the
// kernel maps each CTA to a (level, block) pair); the coupling of level i with i-1 is fused into
// level i's coarse ghosts.  Level i reads buffer (t / 2^i) & 1, so the launch arguments repeat
// with period 2 * 2^(L-1) fine iterations, which is the span captured in the CUDA graph.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbmtree.h"
#include "builder.h"
#include "kernels.h"

using namespace lbm;
extern "C" int lbm_mlp_nparams(void);

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CU(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e__ = (call);                                                                        \
        if (e__ != cudaSuccess) return fail(LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

struct DevLevel {
    int* nbr = nullptr;
    unsigned char* type = nullptr;
    unsigned char* bflag = nullptr;
    int* rec_id = nullptr;
    CellRecDev* recs = nullptr;
    void* f[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    double* lam = nullptr;
    int* blist[2] = {nullptr, nullptr};
    int64_t nlist[2] = {0, 0};
    int* bxyz = nullptr;
    int* blist_all = nullptr;       // every block, for the general kernel alone (far-field relaxation on)
};

struct Constants {
    double w37[37], H37[37 * 15], cs2_37, w21[21], H21[21 * 10];
    Constants() { lattice_constants(w37, H37, &cs2_37, w21, H21); }
};
const Constants& constants() {
    static Constants c;
    return c;
}

std::mutex g_upload_mu;
bool g_uploaded[256] = {false};

bool find_kernels(int lattice, int model, int storage, const int* blk, bool newton_fp32, KernelSet& out) {
    switch (lattice) {
        case LBM_D2Q9: return find_kernels_d2q9(model, storage, blk, out);
        case LBM_D3Q27: return find_kernels_d3q27(model, storage, blk, out);
        case LBM_D2Q37: return find_kernels_d2q37(model, storage, blk, newton_fp32, out);
        case LBM_D2Q13: return find_kernels_d2q13(model, storage, blk, newton_fp32, out);
        case LBM_D2Q21:
            return (model == LBM_BGK || model == LBM_RR) ? find_kernels_d2q21w(model, storage, blk, out)
                                                          : find_kernels_d2q21(model, storage, blk, newton_fp32, out);
    }
    return false;
}
}  // namespace

struct lbm_ctx {
    int dim = 2, device = 0;
    bool host_only = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;        // created by the context (caller passed NULL)
    cudaStream_t side = nullptr;    // general-kernel stream, forked from and joined to `stream`
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int lattice = 0, model = 0, storage = LBM_F64;
    bool params_set = false;
    lbm_collision_params params{};
    FaceSpec faces[6];
    int block[3] = {16, 16, 1};
    BuiltGrid grid;
    bool built = false;
    KernelSet ks;
    int variant = 0;                // compiled step variant in use (lbm_set_variant)
    // host views
    std::vector<int32_t> h_level, h_xyz;
    std::vector<uint8_t> h_type;
    std::vector<int64_t> h_slot;
    std::vector<int64_t> level_first;
    std::vector<int32_t> h_xi;
    // device
    DevLevel dl[MAX_LEVELS];
    int* d_status = nullptr;
    unsigned long long* d_nstat = nullptr;
    double* d_partial = nullptr;
    double* d_out5 = nullptr;
    std::vector<void*> allocs;
    int64_t dev_bytes = 0;
    int64_t t = 0;
    int64_t t_offset = 0;           // fine iterations done before the last remesh
    bool initialized = false;
    int64_t launches = 0;
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    float* d_mlp = nullptr;         // Newton-guess network, weights bf16-rounded (own allocation, kept across grid rebuilds)
    int* d_slot = nullptr;          // slot of every listed cell within its level (device copy of h_slot)
    double* d_rd_lev = nullptr;     // readout scratch (slot order of one level), kept for repeated reads
    double* d_rd_lst = nullptr;     // readout result in listing order
    size_t rd_lev_bytes = 0, rd_lst_bytes = 0;
    std::vector<float> mlp_master;  // its parameters before rounding
    double mlp_m[8] = {0}, mlp_s[8] = {0};
    int64_t total_blocks = 0;

    lbm_allocator alloc_cb{nullptr, nullptr, nullptr};   // caller's device allocator (optional)
    void* dalloc(size_t bytes) {
        void* p = nullptr;
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~size_t(255);              // 256-byte aligned sizes
        if (alloc_cb.alloc) {
            p = alloc_cb.alloc(bytes, alloc_cb.user);
            if (!p) return nullptr;
            if ((uintptr_t)p & 15) {                        // the kernels copy 16-byte rows
                alloc_cb.free(p, alloc_cb.user);
                return nullptr;
            }
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            return nullptr;
        }
        allocs.push_back(p);
        dev_bytes += (int64_t)bytes;
        return p;
    }
    void dfree(void* p) {
        if (alloc_cb.alloc) alloc_cb.free(p, alloc_cb.user);
        else cudaFree(p);
    }
    void release() {
        if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
        for (void* p : allocs) dfree(p);
        allocs.clear();
        dev_bytes = 0;
        for (auto& d : dl) d = DevLevel{};
        d_status = nullptr; d_nstat = nullptr; d_partial = nullptr; d_out5 = nullptr; d_slot = nullptr;
        if (d_rd_lev) cudaFree(d_rd_lev);
        if (d_rd_lst) cudaFree(d_rd_lst);
        d_rd_lev = d_rd_lst = nullptr;
        rd_lev_bytes = rd_lst_bytes = 0;
    }
    int L() const { return grid.n_levels; }
    int64_t period() const { return int64_t(1) << (grid.n_levels - 1); }
    // buffer holding the current state of level i after tt iterations: ceil(tt / 2^i) steps done
    int cur(int i, int64_t tt) const { return int(((tt + (int64_t(1) << i) - 1) >> i) & 1); }
    bool comp() const { return model == LBM_COMP_POLY || model == LBM_COMP_NUMERICAL; }
    int streaming = LBM_STREAM_AB;   // lbm_set_streaming
    std::vector<uint8_t> pending_map;  // level map of the next build (lbm_build_grid_map)
    // what the grid was built from (the remesh rebuilds it with another level map)
    int64_t extent[3] = {1, 1, 1};
    int n_levels_built = 1;
    std::vector<ShapeSpec> solids_built;
    bool weak() const { return model == LBM_BGK || model == LBM_RR || model == LBM_TRT; }
    // kernel-set code of the collision: the public model, with the trace-equilibrated RR as 6
    int kmodel() const { return (model == LBM_RR && params.trace_eq) ? KMODEL_RR_TRACE : model; }
    // far-field relaxation (lbm_set_sponge)
    double sp_c[3] = {0, 0, 0}, sp_r0 = 0, sp_r1 = 1, sp_smax = 0, sp_rho_inf = 1;
    double T0() const {
        if (params.T0 > 0) return params.T0;
        if (lattice == LBM_D2Q21) return 2.0 / 3.0;
        if (lattice == LBM_D2Q13) return 0.5;
        if (lattice == LBM_D2Q37) return constants().cs2_37;
        return 1.0 / 3.0;
    }
};

namespace {

int check_ctx(lbm_ctx* c) {
    if (!c) return fail(LBM_ERR_ARG, "null context");
    return LBM_OK;
}

void fill_args(const lbm_ctx* c, StepArgs& a) {
    std::memset(&a, 0, sizeof(a));
    const int L = c->L();
    a.n_levels = L;
    const int BS = c->grid.BS;
    // tau = nu / theta + 1/2 in each level's units, nu_i = nu_0 / 2^i (Eq. tau_fine_to_coarse);
    // theta = c_s^2 for the weakly compressible models (1/3, 1/2 on D2Q13, 2/3 on D2Q21) and T0
    // for the compressible ones
    const double theta = c->comp() ? c->T0()
                                   : (c->lattice == LBM_D2Q21 ? 2.0 / 3.0 : c->lattice == LBM_D2Q13 ? 0.5 : 1.0 / 3.0);
    for (int i = 0; i < L; ++i) {
        const BuiltLevel& bl = c->grid.levels[i];
        LevelDev& d = a.lv[i];
        d.nb = bl.nb;
        d.ncell = bl.nb * BS;
        d.nbr = c->dl[i].nbr;
        d.type = c->dl[i].type;
        d.bflag = c->dl[i].bflag;
        d.rec_id = c->dl[i].rec_id;
        d.recs = c->dl[i].recs;
        d.f[0] = c->dl[i].f[0]; d.f[1] = c->dl[i].f[1];
        d.g[0] = c->dl[i].g[0]; d.g[1] = c->dl[i].g[1];
        d.lam = c->dl[i].lam;
        for (int k = 0; k < 2; ++k) {
            d.blist[k] = c->dl[i].blist[k];
            d.nlist[k] = c->dl[i].nlist[k];
        }
        if (c->sp_smax > 0) {
            // the far-field relaxation runs in the general kernel only (the interior kernel keeps
            // its register budget): every block goes through the general list
            d.blist[1] = c->dl[i].blist_all;
            d.nlist[0] = 0;
            d.nlist[1] = bl.nb;
        }
        const double nu = c->params.nu0 / double(int64_t(1) << i);
        d.tau = nu / theta + 0.5;
        d.omega = 1.0 / d.tau;
        d.omega_f = (float)d.omega;
        // odd-part rate of the two-relaxation-time collision: (tau - 1/2)(tau_odd - 1/2) = Lambda
        d.omega_m = nu > 0 ? 1.0 / (c->params.trt_magic / (d.tau - 0.5) + 0.5) : d.omega;
        d.omega_m_f = (float)d.omega_m;
        d.bxyz = c->dl[i].bxyz;
        for (int k = 0; k < 3; ++k) d.shape[k] = (int)bl.shape[k];
    }
    ModelDev& m = a.m;
    m.cs2 = theta;
    m.T0 = c->T0();
    m.Cv = 1.0 / (c->params.gamma - 1.0);
    m.rho_ref = c->params.rho_ref > 0 ? c->params.rho_ref : 1.0;
    m.rho_ref_f = (float)m.rho_ref;
    m.inv_rho_ref_f = (float)(1.0 / m.rho_ref);
    {
        const double gref = m.rho_ref * (2.0 * m.Cv - c->dim) * m.T0;
        m.gref_f = (float)gref;
        m.inv_gref_f = gref != 0.0 ? (float)(1.0 / gref) : 0.0f;
    }
    m.sensor_on = c->params.sensor_on;
    m.sensor_A = c->params.sensor_A;
    m.newton_tol = c->params.newton_tol > 0 ? c->params.newton_tol : (c->params.newton_fp32 ? 1e-5 : 1e-12);
    m.newton_max_iter = c->params.newton_max_iter > 0 ? c->params.newton_max_iter : 50;
    m.guess = c->params.guess;
    m.newton_fp32 = c->params.newton_fp32;
    a.aa = c->streaming == LBM_STREAM_AA ? 1 : 0;
    m.sponge_on = c->sp_smax > 0 ? 1 : 0;
    for (int d = 0; d < 3; ++d) m.sp_c[d] = c->sp_c[d];
    m.sp_r0 = c->sp_r0;
    m.sp_r1 = c->sp_r1;
    m.sp_smax = c->sp_smax;
    m.sp_rho_inf = c->sp_rho_inf;
    m.mlp = c->d_mlp;
    for (int k = 0; k < 8; ++k) { m.mlp_m[k] = c->mlp_m[k]; m.mlp_s[k] = c->mlp_s[k]; }
    for (int f = 0; f < 6; ++f) {
        m.faces[f].kind = c->faces[f].kind;
        m.faces[f].rho = c->faces[f].rho;
        for (int d = 0; d < 3; ++d) m.faces[f].u[d] = c->faces[f].u[d];
        m.faces[f].T = c->faces[f].T > 0 ? c->faces[f].T : m.T0;
    }
    a.status = c->d_status;
    a.nstat = c->d_nstat;
}

// arguments of fine iteration t
int64_t iteration_args(const lbm_ctx* c, int64_t t, StepArgs& a) {
    fill_args(c, a);
    const int L = c->L();
    int n = 0;
    int64_t off = 0;
    for (int i = L - 1; i >= 0; --i) {
        if (t % (int64_t(1) << i)) continue;
        if (c->grid.levels[i].nb == 0) continue;
        a.active[n] = i;
        a.block_off[n] = off;
        off += c->grid.levels[i].nb;
        ++n;
    }
    a.block_off[n] = off;
    a.n_active = n;
    for (int k = 0; k < 2; ++k) {
        int64_t o = 0;
        for (int j = 0; j < n; ++j) {
            a.list_off[k][j] = o;
            o += a.lv[a.active[j]].nlist[k];
        }
        a.list_off[k][n] = o;
    }
    for (int i = 0; i < L; ++i) {
        a.rd[i] = int((t >> i) & 1);
        a.sync_fg[i] = (i + 1 < L) && (t % (int64_t(2) << i) == 0);
    }
    return off;
}

// arguments for readout / ledger at the current time: every level, current buffers
int64_t current_args(const lbm_ctx* c, StepArgs& a) {
    fill_args(c, a);
    const int L = c->L();
    int n = 0;
    int64_t off = 0;
    for (int i = L - 1; i >= 0; --i) {
        if (c->grid.levels[i].nb == 0) continue;
        a.active[n] = i;
        a.block_off[n] = off;
        off += c->grid.levels[i].nb;
        ++n;
    }
    a.block_off[n] = off;
    a.n_active = n;
    for (int i = 0; i < L; ++i) a.rd[i] = c->cur(i, c->t);
    if (a.aa) {
        // one buffer: after an even number of iterations it holds layout L1 (own slot qbar = f_q)
        a.rd[0] = 0;
        a.aa_l1 = (c->t % 2 == 0) ? 1 : 0;
    }
    return off;
}

int ready(lbm_ctx* c) {
    if (!c->built) return fail(LBM_ERR_STATE, "grid not built");
    if (c->host_only) return fail(LBM_ERR_STATE, "host-only context (device < 0)");
    if (!c->initialized) return fail(LBM_ERR_STATE, "fields not initialised");
    if (c->params.guess == LBM_GUESS_MLP && !c->d_mlp) return fail(LBM_ERR_STATE, "network guess selected but no network set");
    return LBM_OK;
}

// bfloat16 rounding (nearest even) of a float, as the device conversion does
float bf16_round_host(float v) {
    uint32_t b;
    std::memcpy(&b, &v, 4);
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

// one fine iteration: the general kernel on the side stream beside the interior kernel
void launch_step(lbm_ctx* c, const StepArgs& a) {
    if (a.aa) {                       // in-place streaming: one launch over the single level
        c->ks.aa(a, c->stream);
        return;
    }
    const int64_t nf = a.list_off[0][a.n_active], ng = a.list_off[1][a.n_active];
    if (nf && ng) {
        cudaEventRecord(c->ev_fork, c->stream);
        cudaStreamWaitEvent(c->side, c->ev_fork, 0);
        c->ks.step(a, nf, ng, c->stream, c->side);
        cudaEventRecord(c->ev_join, c->side);
        cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    } else {
        c->ks.step(a, nf, ng, c->stream, c->stream);
    }
}

int launch_iterations(lbm_ctx* c, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        StepArgs a;
        const int64_t nb = iteration_args(c, c->t, a);
        if (nb) {
            launch_step(c, a);
            c->launches += a.aa ? 1 : (a.list_off[0][a.n_active] > 0) + (a.list_off[1][a.n_active] > 0);
        }
        c->t++;
    }
    CU(cudaGetLastError());
    return LBM_OK;
}

int build_graph(lbm_ctx* c) {
    if (c->gexec) return LBM_OK;
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t span = 2 * c->period();
    for (int64_t k = 0; k < span; ++k) {
        StepArgs a;
        const int64_t nb = iteration_args(c, k, a);
        if (nb) launch_step(c, a);
    }
    if (cudaGetLastError() != cudaSuccess) {       // end the capture so the stream stays usable
        cudaGraph_t g2 = nullptr;
        cudaStreamEndCapture(c->stream, &g2);
        if (g2) cudaGraphDestroy(g2);
        return fail(LBM_ERR_CUDA, "launch during graph capture failed");
    }
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return LBM_OK;
}

int launches_per_span(const lbm_ctx* c) {
    int n = 0;
    for (int64_t k = 0; k < 2 * c->period(); ++k) {
        StepArgs a;
        if (iteration_args(c, k, a)) n += a.aa ? 1 : (a.list_off[0][a.n_active] > 0) + (a.list_off[1][a.n_active] > 0);
    }
    return n;
}

}  // namespace

namespace lbm {
// used by noalloc.cu: the arguments of the ledger launch at the current time, the context's
// kernels, stream and device (made current)
int set_error(int code, const std::string& msg) { return fail(code, msg); }

int ledger_launch_args(lbm_ctx* c, StepArgs* a, long long* nblocks, KernelSet* ks, cudaStream_t* s, int* device) {
    if (int r = ready(c)) return r;
    if (c->t % c->period()) return fail(LBM_ERR_STATE, "not at a coarse synchronisation instant");
    CU(cudaSetDevice(c->device));
    *nblocks = current_args(c, *a);
    *ks = c->ks;
    *s = c->stream;
    *device = c->device;
    return LBM_OK;
}
}  // namespace lbm

extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

int lbm_set_allocator(lbm_ctx* c, const lbm_allocator* a) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (c->built) return fail(LBM_ERR_STATE, "the allocator must be set before lbm_build_grid");
    if (a && (!a->alloc || !a->free)) return fail(LBM_ERR_ARG, "allocator needs both alloc and free");
    c->alloc_cb = a ? *a : lbm_allocator{nullptr, nullptr, nullptr};
    return LBM_OK;
}

int lbm_lattice_info(int lattice, int* Q, int* D, int* reach, double* cs2) {
    int q = 0, d = 2, r = 1;
    double c2 = 1.0 / 3.0;
    switch (lattice) {
        case LBM_D2Q9: q = 9; break;
        case LBM_D3Q27: q = 27; d = 3; break;
        case LBM_D2Q13: q = 13; r = 2; c2 = 0.5; break;
        case LBM_D2Q21: q = 21; r = 3; c2 = 2.0 / 3.0; break;
        case LBM_D2Q37: q = 37; r = 3; c2 = constants().cs2_37; break;
        default: return fail(LBM_ERR_ARG, "unknown lattice");
    }
    if (Q) *Q = q;
    if (D) *D = d;
    if (reach) *reach = r;
    if (cs2) *cs2 = c2;
    return LBM_OK;
}

int lbm_create(lbm_ctx** out, int dim, int device, void* stream) {
    if (!out) return fail(LBM_ERR_ARG, "out is null");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(LBM_ERR_ARG, "dim must be 2 or 3");
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(LBM_ERR_OOM, "context allocation");
    c->dim = dim;
    c->device = device;
    c->host_only = device < 0;
    c->stream = (cudaStream_t)stream;
    if (dim == 3) { c->block[0] = 8; c->block[1] = 4; c->block[2] = 4; }
    c->params.gamma = 1.4;
    c->params.rho_ref = 1.0;
    c->params.newton_tol = 1e-12;
    c->params.newton_max_iter = 50;
    c->params.sensor_A = 1.5;
    if (!c->host_only) {
        cudaError_t e = cudaSetDevice(device);
        if (e != cudaSuccess) {
            delete c;
            return fail(LBM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
        }
        if (!c->stream) {
            // a stream of our own: the legacy default stream cannot be captured into a graph
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                delete c;
                return fail(LBM_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            }
            c->own_stream = true;
        }
        // the general blocks go on a high-priority stream: the block scheduler hands them free
        // slots first, so they finish inside the interior sweep instead of after it
        int prio_lo = 0, prio_hi = 0;
        cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
        e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (c->side) cudaStreamDestroy(c->side);
            if (c->ev_fork) cudaEventDestroy(c->ev_fork);
            if (c->own_stream) cudaStreamDestroy(c->stream);
            delete c;
            return fail(LBM_ERR_CUDA, std::string("side stream: ") + cudaGetErrorString(e));
        }
        std::lock_guard<std::mutex> lk(g_upload_mu);
        if (device < 256 && !g_uploaded[device]) {
            const Constants& k = constants();
            e = upload_tables_d2q37(k.w37, k.H37, k.cs2_37);
            if (e == cudaSuccess) e = upload_tables_d2q21(k.w21, k.H21);
            if (e != cudaSuccess) {
                delete c;
                return fail(LBM_ERR_CUDA, std::string("constant upload: ") + cudaGetErrorString(e));
            }
            g_uploaded[device] = true;
        }
    }
    *out = c;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_OK;
    if (!c->host_only) cudaSetDevice(c->device);
    c->release();
    if (c->d_mlp) cudaFree(c->d_mlp);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return LBM_OK;
}

int lbm_set_lattice(lbm_ctx* c, int lattice) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (lattice != LBM_D2Q9 && lattice != LBM_D2Q13 && lattice != LBM_D2Q21 && lattice != LBM_D2Q37 &&
        lattice != LBM_D3Q27)
        return fail(LBM_ERR_ARG, "unknown lattice");
    if ((lattice == LBM_D3Q27) != (c->dim == 3)) return fail(LBM_ERR_ARG, "lattice dimension differs from the context");
    if (c->built) return fail(LBM_ERR_STATE, "lattice must be set before lbm_build_grid");
    c->lattice = lattice;
    return LBM_OK;
}

int lbm_set_collision(lbm_ctx* c, int model, const lbm_collision_params* p) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (model < LBM_BGK || model > LBM_TRT) return fail(LBM_ERR_ARG, "unknown collision model");
    if (c->built) return fail(LBM_ERR_STATE, "collision model must be set before lbm_build_grid");
    if (model == LBM_TRT && (!p || p->nu0 <= 0))
        return fail(LBM_ERR_ARG, "the two-relaxation-time collision needs a positive viscosity");
    if (p) {
        if (p->nu0 < 0) return fail(LBM_ERR_ARG, "negative viscosity");
        if (p->trace_eq && model != LBM_RR) return fail(LBM_ERR_ARG, "trace equilibration applies to LBM_RR");
        if (p->gamma <= 1.0 && model >= LBM_COMP_POLY) return fail(LBM_ERR_ARG, "gamma must exceed 1");
        if (p->guess < 0 || p->guess > LBM_GUESS_MLP) return fail(LBM_ERR_ARG, "unknown Newton guess");
        if (p->newton_fp32 && p->newton_tol > 0 && p->newton_tol < 1e-6)
            return fail(LBM_ERR_ARG, "an FP32 Newton solve cannot reach a tolerance below 1e-6 (use 1e-5)");
        c->params = *p;
        if (c->params.gamma <= 1.0) c->params.gamma = 1.4;
        if (c->params.rho_ref <= 0) c->params.rho_ref = 1.0;
        if (c->params.trt_magic <= 0) c->params.trt_magic = 0.25;
    } else {
        c->params = lbm_collision_params{};
        c->params.gamma = 1.4;
        c->params.rho_ref = 1.0;
        c->params.trt_magic = 0.25;
    }
    c->model = model;
    c->params_set = true;
    return LBM_OK;
}

int lbm_set_guess(lbm_ctx* c, int guess) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (guess < LBM_GUESS_WARM || guess > LBM_GUESS_MLP) return fail(LBM_ERR_ARG, "unknown Newton guess");
    c->params.guess = guess;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return LBM_OK;
}

int lbm_set_newton_precision(lbm_ctx* c, int fp32, double tol) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (fp32 && tol > 0 && tol < 1e-6)
        return fail(LBM_ERR_ARG, "an FP32 Newton solve cannot reach a tolerance below 1e-6 (use 1e-5)");
    c->params.newton_fp32 = fp32 ? 1 : 0;
    c->params.newton_tol = tol;
    if (c->built) {
        // the two precisions are separate kernel sets (D2Q21); keep the variant in use
        KernelSet ks;
        if (find_kernels(c->lattice, c->kmodel(), c->storage, c->block, fp32 != 0, ks)) {
            ks.step = ks.variant[c->variant < ks.n_variants ? c->variant : 0];
            c->ks = ks;
        }
    }
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return LBM_OK;
}

int lbm_set_sponge(lbm_ctx* c, const double centre[3], double r0, double r1, double sigma_max, double rho_inf) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!centre) return fail(LBM_ERR_ARG, "null centre");
    if (!(r1 > r0) || !(sigma_max >= 0.0 && sigma_max <= 1.0) || !(rho_inf > 0.0))
        return fail(LBM_ERR_ARG, "need r1 > r0, sigma_max in [0, 1] and rho_inf > 0");
    if (c->params_set && c->comp() && sigma_max > 0)
        return fail(LBM_ERR_UNSUPPORTED, "the far-field relaxation is built for the weakly compressible models");
    for (int d = 0; d < 3; ++d) c->sp_c[d] = centre[d];
    c->sp_r0 = r0;
    c->sp_r1 = r1;
    c->sp_smax = sigma_max;
    c->sp_rho_inf = rho_inf;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return LBM_OK;
}

int lbm_set_streaming(lbm_ctx* c, int mode) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (mode != LBM_STREAM_AB && mode != LBM_STREAM_AA) return fail(LBM_ERR_ARG, "unknown streaming mode");
    if (c->built) return fail(LBM_ERR_STATE, "streaming must be set before lbm_build_grid");
    c->streaming = mode;
    return LBM_OK;
}

int lbm_set_precision(lbm_ctx* c, int storage) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (storage != LBM_F64 && storage != LBM_F32 && storage != LBM_F16DEV) return fail(LBM_ERR_ARG, "unknown storage");
    if (c->built) return fail(LBM_ERR_STATE, "precision must be set before lbm_build_grid");
    c->storage = storage;
    return LBM_OK;
}

int lbm_set_boundary(lbm_ctx* c, int face, int kind, const double* v) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (face < 0 || face > 5) return fail(LBM_ERR_ARG, "face out of range");
    if (kind < LBM_PERIODIC || kind > LBM_WALL) return fail(LBM_ERR_ARG, "unknown boundary kind");
    if ((kind == LBM_EQ_DIRICHLET || kind == LBM_EQ_DIRICHLET_RHO) && !v) return fail(LBM_ERR_ARG, "Dirichlet values missing");
    if (c->built) return fail(LBM_ERR_STATE, "boundaries must be set before lbm_build_grid");
    FaceSpec& f = c->faces[face];
    f.kind = kind;
    if (v) { f.rho = v[0]; f.u[0] = v[1]; f.u[1] = v[2]; f.u[2] = v[3]; f.T = v[4]; }
    else { f.rho = 1.0; f.u[0] = f.u[1] = f.u[2] = 0.0; f.T = 0.0; }
    if (kind == LBM_WALL && !(f.rho > 0)) return fail(LBM_ERR_ARG, "wall density must be positive");
    return LBM_OK;
}

int lbm_set_block(lbm_ctx* c, int bx, int by, int bz) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (c->built) return fail(LBM_ERR_STATE, "block shape must be set before lbm_build_grid");
    if (bx < 2 || by < 2 || bz < 1 || (c->dim == 2 && bz != 1) || bx * by * bz > 1024)
        return fail(LBM_ERR_ARG, "bad block shape");
    c->block[0] = bx; c->block[1] = by; c->block[2] = bz;
    return LBM_OK;
}

int lbm_build_grid(lbm_ctx* c, const int64_t extent[3], int n_levels, const lbm_box* boxes, int n_boxes,
                   const lbm_shape* solids, int n_solids) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!extent || (n_boxes > 0 && !boxes) || (n_solids > 0 && !solids)) return fail(LBM_ERR_ARG, "null array");
    if (!c->lattice || !c->params_set) return fail(LBM_ERR_STATE, "set lattice and collision model first");
    if (c->built) return fail(LBM_ERR_STATE, "grid already built");
    const bool weak = c->weak();
    if ((weak && !(c->lattice == LBM_D2Q9 || c->lattice == LBM_D3Q27 || c->lattice == LBM_D2Q21 ||
                   c->lattice == LBM_D2Q13)) ||
        ((c->model == LBM_TRT || c->kmodel() == KMODEL_RR_TRACE) &&
         !(c->lattice == LBM_D2Q9 || c->lattice == LBM_D3Q27)) ||
        (c->model == LBM_COMP_POLY && c->lattice != LBM_D2Q37) ||
        (c->model == LBM_COMP_NUMERICAL && c->lattice != LBM_D2Q13 && c->lattice != LBM_D2Q21 &&
         c->lattice != LBM_D2Q37))
        return fail(LBM_ERR_UNSUPPORTED, "lattice/model combination not built");
    if (c->sp_smax > 0 && !weak) return fail(LBM_ERR_UNSUPPORTED, "the far-field relaxation is built for the weakly compressible models");
    if (c->streaming == LBM_STREAM_AA) {
        if (n_levels != 1) return fail(LBM_ERR_UNSUPPORTED, "AA streaming is built for single-level grids");
        for (int f = 0; f < 2 * c->dim; ++f)
            if (c->faces[f].kind == LBM_EQ_DIRICHLET_RHO || c->faces[f].kind == LBM_NEUMANN)
                return fail(LBM_ERR_UNSUPPORTED, "AA streaming takes periodic, wall and imposed-equilibrium faces");
    }
    for (int f = 0; f < 6; ++f)
        if (c->faces[f].kind == LBM_WALL && !weak &&
            (c->faces[f].u[0] != 0.0 || c->faces[f].u[1] != 0.0 || c->faces[f].u[2] != 0.0))
            return fail(LBM_ERR_UNSUPPORTED, "moving walls are built for the weakly compressible models");
    if (!find_kernels(c->lattice, c->kmodel(), c->storage, c->block, c->params.newton_fp32 != 0, c->ks))
        return fail(LBM_ERR_UNSUPPORTED, "no kernel for this lattice/model/storage/block shape");
    if (c->streaming == LBM_STREAM_AA && !c->ks.aa)
        return fail(LBM_ERR_UNSUPPORTED, "AA streaming is compiled for D2Q9 and D3Q27 (BGK, RR) and D2Q37 (polynomial DDF)");
    GridInput in;
    in.dim = c->dim;
    for (int d = 0; d < 3; ++d) in.extent[d] = extent[d];
    in.n_levels = n_levels;
    for (int k = 0; k < n_boxes; ++k) {
        BoxSpec b;
        b.level = boxes[k].level;
        for (int d = 0; d < 3; ++d) { b.lo[d] = boxes[k].lo[d]; b.hi[d] = boxes[k].hi[d]; }
        in.boxes.push_back(b);
    }
    for (int k = 0; k < n_solids; ++k) {
        ShapeSpec s;
        s.kind = solids[k].kind;
        std::memcpy(s.p, solids[k].p, sizeof(s.p));
        in.solids.push_back(s);
    }
    for (int f = 0; f < 6; ++f) in.faces[f] = c->faces[f];
    for (int d = 0; d < 3; ++d) in.block[d] = c->block[d];
    in.lattice = c->lattice;
    in.level_map = std::move(c->pending_map);
    c->pending_map.clear();
    for (int d = 0; d < 3; ++d) c->extent[d] = extent[d];
    c->n_levels_built = n_levels;
    c->solids_built = in.solids;
    std::string err;
    try {
        err = build_grid(in, c->grid);
    } catch (const std::bad_alloc&) {
        return fail(LBM_ERR_OOM, "host allocation in the grid builder");
    } catch (...) {
        return fail(LBM_ERR_GRID, "grid builder failed");
    }
    if (!err.empty()) return fail(LBM_ERR_GRID, err);
    const int BS = c->grid.BS;
    c->h_level.clear(); c->h_xyz.clear(); c->h_type.clear(); c->h_slot.clear(); c->level_first.clear();
    for (int i = 0; i < c->L(); ++i) {
        const BuiltLevel& lv = c->grid.levels[i];
        c->level_first.push_back((int64_t)c->h_type.size());
        for (int64_t b = 0; b < lv.nb; ++b)
            for (int l = 0; l < BS; ++l) {
                const uint8_t t = lv.type[b * BS + l];
                if (t == C_ABSENT) continue;
                const int lx = l % c->block[0], ly = (l / c->block[0]) % c->block[1], lz = l / (c->block[0] * c->block[1]);
                c->h_level.push_back(i);
                c->h_xyz.push_back(lv.bxyz[3 * b] * c->block[0] + lx);
                c->h_xyz.push_back(lv.bxyz[3 * b + 1] * c->block[1] + ly);
                c->h_xyz.push_back(lv.bxyz[3 * b + 2] * c->block[2] + lz);
                c->h_type.push_back(t);
                c->h_slot.push_back(b * BS + l);
            }
    }
    c->level_first.push_back((int64_t)c->h_type.size());
    c->h_xi.clear();
    for (int q = 0; q < c->grid.lat.Q; ++q)
        for (int d = 0; d < 3; ++d) c->h_xi.push_back(c->grid.lat.xi[q][d]);
    c->built = true;
    if (c->host_only) return LBM_OK;
    CU(cudaSetDevice(c->device));
    const int Q = c->grid.lat.Q;
    const size_t es = c->storage == LBM_F64 ? 8 : c->storage == LBM_F32 ? 4 : 2;
    const bool has_g = c->comp();
    const bool has_lam = c->model == LBM_COMP_NUMERICAL;
    c->total_blocks = 0;
    for (int i = 0; i < c->L(); ++i) {
        const BuiltLevel& lv = c->grid.levels[i];
        DevLevel& d = c->dl[i];
        const int64_t ncell = lv.nb * BS;
        if ((ncell + BS) * int64_t(Q) >= (int64_t(1) << 32)) {
            c->release();
            c->built = false;
            return fail(LBM_ERR_GRID, "level " + std::to_string(i) + " too large for 32-bit population offsets");
        }
        c->total_blocks += lv.nb;
        d.nbr = (int*)c->dalloc(lv.nbr.size() * 4);
        d.type = (unsigned char*)c->dalloc(lv.type.size());
        d.bflag = (unsigned char*)c->dalloc(lv.bflag.size());
        d.rec_id = (int*)c->dalloc(lv.rec_id.size() * 4);
        d.recs = (CellRecDev*)c->dalloc(lv.recs.size() * sizeof(CellRecDev));
        // one extra block of zero populations stands in for missing neighbour blocks
        // AA streaming keeps one population buffer (both pointers name it)
        const int nbuf = c->streaming == LBM_STREAM_AA ? 1 : 2;
        for (int k = 0; k < nbuf; ++k) {
            d.f[k] = c->dalloc(size_t(Q) * (ncell + BS) * es);
            if (has_g) d.g[k] = c->dalloc(size_t(Q) * (ncell + BS) * es);
        }
        if (nbuf == 1) {
            d.f[1] = d.f[0];
            d.g[1] = d.g[0];
        }
        if (has_lam) d.lam = (double*)c->dalloc(size_t(2) * 8 * ncell * 8);
        if (!d.nbr || !d.type || !d.bflag || !d.rec_id || !d.recs || !d.f[0] || !d.f[1] ||
            (has_g && (!d.g[0] || !d.g[1])) || (has_lam && !d.lam)) {
            c->release();
            c->built = false;
            return fail(LBM_ERR_OOM, "device allocation of level " + std::to_string(i));
        }
        CU(cudaMemcpy(d.nbr, lv.nbr.data(), lv.nbr.size() * 4, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d.type, lv.type.data(), lv.type.size(), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d.bflag, lv.bflag.data(), lv.bflag.size(), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d.rec_id, lv.rec_id.data(), lv.rec_id.size() * 4, cudaMemcpyHostToDevice));
        d.bxyz = (int*)c->dalloc(lv.bxyz.size() * 4);
        if (!d.bxyz) {
            c->release();
            c->built = false;
            return fail(LBM_ERR_OOM, "device allocation of the block coordinates");
        }
        CU(cudaMemcpy(d.bxyz, lv.bxyz.data(), lv.bxyz.size() * 4, cudaMemcpyHostToDevice));
        // list 0 entries: 2 * block + 1 for streaming blocks (cell types read), 2 * block for
        // simple blocks; list 1: the general blocks
        std::vector<int32_t> lists[2];
        for (int64_t b = 0; b < lv.nb; ++b) {
            if (lv.bflag[b]) lists[0].push_back((int32_t)(4 * b + (lv.bflag[b] >= 2 ? 1 : 0) + (lv.bflag[b] == 3 ? 2 : 0)));
            else lists[1].push_back((int32_t)b);
        }
        for (int k = 0; k < 2; ++k) {
            d.nlist[k] = (int64_t)lists[k].size();
            d.blist[k] = (int*)c->dalloc(lists[k].size() * 4);
            if (!d.blist[k]) {
                c->release();
                c->built = false;
                return fail(LBM_ERR_OOM, "device allocation of the block lists");
            }
            if (!lists[k].empty()) CU(cudaMemcpy(d.blist[k], lists[k].data(), lists[k].size() * 4, cudaMemcpyHostToDevice));
        }
        if (!lv.recs.empty())
            CU(cudaMemcpy(d.recs, lv.recs.data(), lv.recs.size() * sizeof(CellRecDev), cudaMemcpyHostToDevice));
        {
            std::vector<int32_t> all(lv.nb);
            for (int64_t b = 0; b < lv.nb; ++b) all[b] = (int32_t)b;
            d.blist_all = (int*)c->dalloc(std::max<size_t>(all.size(), 1) * 4);
            if (!d.blist_all) {
                c->release();
                c->built = false;
                return fail(LBM_ERR_OOM, "device allocation of the block lists");
            }
            if (!all.empty()) CU(cudaMemcpy(d.blist_all, all.data(), all.size() * 4, cudaMemcpyHostToDevice));
        }
    }
    c->d_status = (int*)c->dalloc(sizeof(int));
    c->d_nstat = (unsigned long long*)c->dalloc(19 * sizeof(unsigned long long));
    c->d_partial = (double*)c->dalloc(size_t(c->total_blocks + 1) * 5 * sizeof(double));
    c->d_out5 = (double*)c->dalloc(5 * sizeof(double));
    if (!c->d_status || !c->d_nstat || !c->d_partial || !c->d_out5) {
        c->release();
        c->built = false;
        return fail(LBM_ERR_OOM, "device allocation");
    }
    CU(cudaMemset(c->d_status, 0, sizeof(int)));
    CU(cudaMemset(c->d_nstat, 0, 19 * sizeof(unsigned long long)));
    return LBM_OK;
}

namespace {

// cell (type, slot) of a built grid at level i and level coordinates c (periodic axes wrap)
uint8_t grid_cell(const BuiltGrid& g, int i, const int64_t* c, int64_t* slot) {
    const BuiltLevel& lv = g.levels[i];
    int64_t w[3] = {c[0], c[1], c[2]};
    for (int d = 0; d < g.dim; ++d) {
        if (w[d] < 0 || w[d] >= lv.shape[d]) {
            if (!g.periodic[d]) return C_ABSENT;
            w[d] = ((w[d] % lv.shape[d]) + lv.shape[d]) % lv.shape[d];
        }
    }
    int64_t bc[3], l[3];
    for (int d = 0; d < 3; ++d) { bc[d] = w[d] / g.block[d]; l[d] = w[d] % g.block[d]; }
    const int32_t b = lv.bindex[(bc[2] * lv.bgrid[1] + bc[1]) * lv.bgrid[0] + bc[0]];
    if (b < 0) return C_ABSENT;
    *slot = int64_t(b) * g.BS + (l[2] * g.block[1] + l[1]) * g.block[0] + l[0];
    return lv.type[*slot];
}

// Sources of the remesh transfer (Sec. 8): a new cell takes the old conserved state at the same
// level and place (coarse ghosts with their unknowns coalesced; a fine ghost stands for its
// coarse-ghost parent), else the old coarser cell holding it (uniform explosion), else the mean
// of its children resolved the same way (coalescence).  Entries (old level << 40 | slot, weight).
bool transfer_sources(const BuiltGrid& old, int i, const int64_t* c, double w,
                      std::vector<std::pair<long long, double>>& out) {
    int64_t s;
    const uint8_t t = grid_cell(old, i, c, &s);
    if (t == C_FLUID || t == C_BC || t == C_CGHOST) {
        out.push_back({((long long)i << 40) | s, w});
        return true;
    }
    if (t == C_SOLID) return true;                          // no fluid state there
    if (t == C_FGHOST) {
        const int64_t p[3] = {c[0] >> 1, old.dim > 1 ? c[1] >> 1 : c[1], old.dim > 2 ? c[2] >> 1 : c[2]};
        if (grid_cell(old, i + 1, p, &s) != C_CGHOST) return false;
        out.push_back({((long long)(i + 1) << 40) | s, w});
        return true;
    }
    bool finer = false;                                      // covered by an old finer level?
    for (int j = 0; j < i && !finer; ++j) {
        const int sh = i - j;
        const int64_t cj[3] = {c[0] << sh, old.dim > 1 ? c[1] << sh : c[1], old.dim > 2 ? c[2] << sh : c[2]};
        int64_t s2;
        finer = grid_cell(old, j, cj, &s2) != C_ABSENT;
    }
    if (finer) {
        const int64_t ch[3] = {2 * c[0], old.dim > 1 ? 2 * c[1] : c[1], old.dim > 2 ? 2 * c[2] : c[2]};
        {
            const int nk = 1 << old.dim;
            for (int k = 0; k < nk; ++k) {
                const int64_t cc[3] = {ch[0] + (k & 1), ch[1] + ((k >> 1) & 1), ch[2] + ((k >> 2) & 1)};
                if (!transfer_sources(old, i - 1, cc, w / nk, out)) return false;
            }
            return true;
        }
    }
    for (int j = i + 1; j < old.n_levels; ++j) {             // an old coarser cell holds it
        const int sh = j - i;
        const int64_t p[3] = {c[0] >> sh, old.dim > 1 ? c[1] >> sh : c[1], old.dim > 2 ? c[2] >> sh : c[2]};
        const uint8_t tj = grid_cell(old, j, p, &s);
        if (tj == C_ABSENT) continue;
        if (tj == C_FLUID || tj == C_BC || tj == C_CGHOST) {
            out.push_back({((long long)j << 40) | s, w});
            return true;
        }
        return transfer_sources(old, j, p, w, out);
    }
    return false;
}

}  // namespace

int lbm_build_grid_map(lbm_ctx* c, const int64_t extent[3], int n_levels, const uint8_t* level_map,
                       const lbm_shape* solids, int n_solids) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!extent || !level_map) return fail(LBM_ERR_ARG, "null array");
    if (c->built) return fail(LBM_ERR_STATE, "grid already built");
    int64_t n0 = 1;
    for (int d = 0; d < c->dim; ++d) {
        if (extent[d] <= 0) return fail(LBM_ERR_ARG, "non-positive extent");
        n0 *= extent[d];
    }
    c->pending_map.assign(level_map, level_map + n0);
    return lbm_build_grid(c, extent, n_levels, nullptr, 0, solids, n_solids);
}

int lbm_grade_level_map(int dim, const int64_t extent[3], int n_levels, int lattice, const int periodic[3],
                        uint8_t* level_map) {
    if ((dim != 2 && dim != 3) || !extent || !periodic || !level_map) return fail(LBM_ERR_ARG, "bad arguments");
    if (n_levels < 1 || n_levels > MAX_LEVELS) return fail(LBM_ERR_ARG, "n_levels out of range");
    int Q = 0, D = 0, R = 0;
    double cs2 = 0;
    if (lbm_lattice_info(lattice, &Q, &D, &R, &cs2) != LBM_OK || D != dim) return fail(LBM_ERR_ARG, "unknown lattice");
    for (int d = 0; d < dim; ++d)
        if (extent[d] <= 0 || extent[d] % (int64_t(1) << (n_levels - 1))) return fail(LBM_ERR_ARG, "extent not divisible by 2^(n_levels-1)");
    bool per[3] = {periodic[0] != 0, periodic[1] != 0, periodic[2] != 0};
    grade_level_map(dim, extent, n_levels, 3 * R + 1, per, level_map);
    return LBM_OK;
}

int lbm_amr_level_map(lbm_ctx* c, double threshold, const uint8_t* fixed_map, uint8_t* level_map) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!level_map) return fail(LBM_ERR_ARG, "null output");
    if (int r = ready(c)) return r;
    const int L = c->L();
    const int64_t* e = c->extent;
    const int64_t n0 = e[0] * (c->dim > 1 ? e[1] : 1) * (c->dim > 2 ? e[2] : 1);
    for (int64_t k = 0; k < n0; ++k) level_map[k] = fixed_map ? std::min<uint8_t>(fixed_map[k], (uint8_t)(L - 1)) : (uint8_t)(L - 1);
    // kinetic sensor of every cell (pre-collision state), level by level
    StepArgs a;
    current_args(c, a);
    size_t need = 0;
    for (int i = 0; i < L; ++i) need = std::max(need, size_t(c->grid.levels[i].nb) * c->grid.BS * sizeof(double));
    double* d = nullptr;
    if (cudaMalloc(&d, need ? need : 8) != cudaSuccess) return fail(LBM_ERR_OOM, "sensor buffer");
    std::vector<double> eps;
    int status = LBM_OK;
    for (int i = 0; i < L && status == LBM_OK; ++i) {
        const BuiltLevel& lv = c->grid.levels[i];
        const int64_t ncell = lv.nb * c->grid.BS;
        if (!ncell) continue;
        c->ks.read(a, i, 7, d, c->stream);
        eps.resize(ncell);
        if (cudaMemcpyAsync(eps.data(), d, ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            status = fail(LBM_ERR_CUDA, "sensor readout");
            break;
        }
        const int64_t f = int64_t(1) << i;
        for (int64_t slot = 0; slot < ncell; ++slot) {
            const uint8_t t = lv.type[slot];
            if (!(t == C_FLUID || t == C_BC) || !(eps[slot] > threshold)) continue;
            const int64_t b = slot / c->grid.BS, l = slot % c->grid.BS;
            const int64_t x = lv.bxyz[3 * b] * c->block[0] + l % c->block[0];
            const int64_t y = lv.bxyz[3 * b + 1] * c->block[1] + (l / c->block[0]) % c->block[1];
            const int64_t z = lv.bxyz[3 * b + 2] * c->block[2] + l / (c->block[0] * c->block[1]);
            // every finest cell under a flagged cell wants the finest level
            for (int64_t zz = (c->dim > 2 ? z * f : 0); zz < (c->dim > 2 ? (z + 1) * f : 1); ++zz)
                for (int64_t yy = y * f; yy < (y + 1) * f; ++yy)
                    for (int64_t xx = x * f; xx < (x + 1) * f; ++xx) level_map[(zz * e[1] + yy) * e[0] + xx] = 0;
        }
    }
    cudaFree(d);
    if (status != LBM_OK) return status;
    bool per[3] = {c->grid.periodic[0], c->grid.periodic[1], c->grid.periodic[2]};
    grade_level_map(c->dim, e, L, 3 * c->grid.lat.R + 1, per, level_map);
    return LBM_OK;
}

int lbm_remesh(lbm_ctx* c, const uint8_t* level_map) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!level_map) return fail(LBM_ERR_ARG, "null level map");
    if (int r = ready(c)) return r;
    if (c->streaming != LBM_STREAM_AB) return fail(LBM_ERR_UNSUPPORTED, "remesh needs two-buffer streaming");
    if (c->t % c->period()) return fail(LBM_ERR_STATE, "not at a coarse synchronisation instant");
    if (int r = lbm_sync(c)) return r;
    const int Q = c->grid.lat.Q;
    const bool has_g = c->comp(), has_lam = c->model == LBM_COMP_NUMERICAL;
    const int ncomp = Q + (has_g ? Q : 0) + (has_lam ? 8 : 0);
    const int Lold = c->L();
    // 1. the old conserved state, per level, slot-indexed: f, g, lambda
    StepArgs a;
    current_args(c, a);
    TransferSrc src{};
    std::vector<double*> olds(Lold, nullptr);
    auto free_olds = [&]() { for (double* p : olds) if (p) cudaFree(p); };
    for (int i = 0; i < Lold; ++i) {
        const int64_t ncell = c->grid.levels[i].nb * c->grid.BS;
        if (cudaMalloc(&olds[i], size_t(ncomp) * std::max<int64_t>(ncell, 1) * 8) != cudaSuccess) {
            free_olds();
            return fail(LBM_ERR_OOM, "remesh staging");
        }
        if (ncell) {
            c->ks.read(a, i, 4, olds[i], c->stream);
            if (has_g) c->ks.read(a, i, 5, olds[i] + size_t(Q) * ncell, c->stream);
            if (has_lam) c->ks.read(a, i, 6, olds[i] + size_t(Q + (has_g ? Q : 0)) * ncell, c->stream);
        }
        src.ptr[i] = olds[i];
        src.ncell[i] = ncell;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) { free_olds(); return fail(LBM_ERR_CUDA, "remesh readout"); }
    // 2. the new grid, from the same settings and solids
    BuiltGrid old = std::move(c->grid);
    const int64_t fine_it = c->t + c->t_offset, launches = c->launches;
    c->release();
    c->built = false;
    c->initialized = false;
    std::vector<lbm_shape> sh(c->solids_built.size());
    for (size_t k = 0; k < sh.size(); ++k) {
        sh[k].kind = c->solids_built[k].kind;
        std::memcpy(sh[k].p, c->solids_built[k].p, sizeof(sh[k].p));
    }
    int64_t ext[3] = {c->extent[0], c->extent[1], c->extent[2]};
    if (int r = lbm_build_grid_map(c, ext, c->n_levels_built, level_map, sh.empty() ? nullptr : sh.data(), (int)sh.size())) {
        free_olds();
        return r;                  // the context is left unbuilt; the message says why
    }
    // 3. transfer rows per new level, then the state into the new buffers
    StepArgs na;
    fill_args(c, na);
    int status = LBM_OK;
    for (int i = 0; i < c->L() && status == LBM_OK; ++i) {
        const BuiltLevel& lv = c->grid.levels[i];
        const int64_t rows = lv.nb * c->grid.BS;
        if (!rows) continue;
        std::vector<long long> rowptr(rows + 1, 0), col;
        std::vector<double> w;
        std::vector<std::pair<long long, double>> ent;
        for (int64_t slot = 0; slot < rows && status == LBM_OK; ++slot) {
            const uint8_t t = lv.type[slot];
            if (t != C_ABSENT && t != C_SOLID) {
                const int64_t b = slot / c->grid.BS, l = slot % c->grid.BS;
                const int64_t cc[3] = {lv.bxyz[3 * b] * c->block[0] + l % c->block[0],
                                       lv.bxyz[3 * b + 1] * c->block[1] + (l / c->block[0]) % c->block[1],
                                       lv.bxyz[3 * b + 2] * c->block[2] + l / (c->block[0] * c->block[1])};
                ent.clear();
                if (!transfer_sources(old, i, cc, 1.0, ent)) status = fail(LBM_ERR_GRID, "remesh: a new cell has no old state");
                for (auto& e : ent) { col.push_back(e.first); w.push_back(e.second); }
            }
            rowptr[slot + 1] = (long long)col.size();
        }
        if (status != LBM_OK) break;
        long long *d_row = nullptr, *d_col = nullptr;
        double *d_w = nullptr, *d_new = nullptr;
        const size_t ncol = std::max<size_t>(col.size(), 1);
        if (cudaMalloc(&d_row, rowptr.size() * 8) != cudaSuccess || cudaMalloc(&d_col, ncol * 8) != cudaSuccess ||
            cudaMalloc(&d_w, ncol * 8) != cudaSuccess || cudaMalloc(&d_new, size_t(ncomp) * rows * 8) != cudaSuccess) {
            status = fail(LBM_ERR_OOM, "remesh transfer");
        } else {
            cudaMemcpy(d_row, rowptr.data(), rowptr.size() * 8, cudaMemcpyHostToDevice);
            if (!col.empty()) {
                cudaMemcpy(d_col, col.data(), col.size() * 8, cudaMemcpyHostToDevice);
                cudaMemcpy(d_w, w.data(), w.size() * 8, cudaMemcpyHostToDevice);
            }
            launch_transfer(d_row, d_col, d_w, rows, src, ncomp, d_new, c->stream);
            c->ks.load_state(na, i, d_new, c->stream);
            if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
                status = fail(LBM_ERR_CUDA, "remesh transfer kernels");
        }
        cudaFree(d_row); cudaFree(d_col); cudaFree(d_w); cudaFree(d_new);
    }
    free_olds();
    if (status != LBM_OK) return status;
    for (int i = 1; i < c->L(); ++i) c->ks.remesh_corners(na, i, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(LBM_ERR_CUDA, "remesh corner kernels");
    c->t = 0;
    c->t_offset = fine_it;        // the schedule restarts; the counter of the stats goes on
    c->launches = launches;
    c->initialized = true;
    return LBM_OK;
}

int lbm_cells(lbm_ctx* c, int64_t* n, const int32_t** level, const int32_t** xyz, const uint8_t** type) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!c->built) return fail(LBM_ERR_STATE, "grid not built");
    if (n) *n = (int64_t)c->h_type.size();
    if (level) *level = c->h_level.data();
    if (xyz) *xyz = c->h_xyz.data();
    if (type) *type = c->h_type.data();
    return LBM_OK;
}

int lbm_velocities(lbm_ctx* c, int* Q, const int32_t** xi) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!c->built) return fail(LBM_ERR_STATE, "grid not built");
    if (Q) *Q = c->grid.lat.Q;
    if (xi) *xi = c->h_xi.data();
    return LBM_OK;
}

// device copy of the listing -> slot table (made on first use, freed with the grid)
int ensure_slots(lbm_ctx* c) {
    if (c->d_slot) return LBM_OK;
    const int64_t n = (int64_t)c->h_slot.size();
    std::vector<int32_t> s32(n);
    for (int64_t k = 0; k < n; ++k) s32[k] = (int32_t)c->h_slot[k];
    c->d_slot = (int*)c->dalloc(size_t(n) * 4);
    if (!c->d_slot) return fail(LBM_ERR_OOM, "slot table");
    CU(cudaMemcpy(c->d_slot, s32.data(), size_t(n) * 4, cudaMemcpyHostToDevice));
    return LBM_OK;
}

int lbm_init_fields(lbm_ctx* c, const double* rho, const double* u, const double* T) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!c->built) return fail(LBM_ERR_STATE, "grid not built");
    if (c->host_only) return fail(LBM_ERR_STATE, "host-only context");
    const bool comp = c->comp();
    if (!rho || !u || (comp && !T)) return fail(LBM_ERR_ARG, "null field array");
    CU(cudaSetDevice(c->device));
    const int64_t n = (int64_t)c->h_type.size();
    const int BS = c->grid.BS;
    StepArgs a;
    fill_args(c, a);
    if (int r = ensure_slots(c)) return r;
    // the fields in listing order on the device (one copy per field), then per level moved to
    // slot order and turned into equilibria
    const int nc = 1 + c->dim + (comp ? 1 : 0);
    int64_t maxcell = 0;
    for (int i = 0; i < c->L(); ++i) maxcell = std::max<int64_t>(maxcell, c->grid.levels[i].nb * BS);
    double *d_list = nullptr, *d_lev = nullptr;
    int rc = LBM_OK;
    if (cudaMalloc(&d_list, size_t(nc) * n * 8) != cudaSuccess || cudaMalloc(&d_lev, size_t(5) * maxcell * 8) != cudaSuccess) {
        rc = fail(LBM_ERR_OOM, "initialisation staging");
    } else if (cudaMemcpyAsync(d_list, rho, size_t(n) * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
               cudaMemcpyAsync(d_list + n, u, size_t(c->dim) * n * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
               (comp && cudaMemcpyAsync(d_list + (1 + c->dim) * n, T, size_t(n) * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)) {
        rc = fail(LBM_ERR_CUDA, "initialisation upload");
    }
    for (int i = 0; i < c->L() && rc == LBM_OK; ++i) {
        const int64_t ncell = c->grid.levels[i].nb * BS;
        if (!ncell) continue;
        const int64_t f0 = c->level_first[i], cnt = c->level_first[i + 1] - f0;
        double* pr = d_lev;
        double* pu = d_lev + ncell;
        double* pT = d_lev + 4 * ncell;
        cudaMemsetAsync(d_lev, 0, size_t(5) * ncell * 8, c->stream);
        launch_scatter(c->d_slot + f0, cnt, d_list + f0, n, 1, pr, ncell, c->stream);
        launch_scatter(c->d_slot + f0, cnt, d_list + n + f0, n, c->dim, pu, ncell, c->stream);
        if (comp) launch_scatter(c->d_slot + f0, cnt, d_list + (1 + c->dim) * n + f0, n, 1, pT, ncell, c->stream);
        c->ks.init(a, i, pr, pu, pT, c->stream);
        cudaError_t e = cudaStreamSynchronize(c->stream);      // the staging buffer is reused per level
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) rc = fail(LBM_ERR_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
    }
    cudaFree(d_list);
    cudaFree(d_lev);
    if (rc) return rc;
    int st = 0;
    CU(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemset(c->d_status, 0, sizeof(int)));
    CU(cudaMemset(c->d_nstat, 0, 19 * sizeof(unsigned long long)));
    c->t = 0;
    c->t_offset = 0;
    c->launches = 0;
    c->initialized = true;
    if (st) return fail(st, "initialisation: a Newton solve did not converge");
    return LBM_OK;
}

int lbm_step_fine(lbm_ctx* c, int64_t n) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (int r = ready(c)) return r;
    if (n < 0) return fail(LBM_ERR_ARG, "negative step count");
    return launch_iterations(c, n);
}

int lbm_variants(lbm_ctx* c, int* n, int* minb) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!c->built) return fail(LBM_ERR_STATE, "grid not built");
    if (n) *n = c->ks.n_variants;
    if (minb)
        for (int k = 0; k < c->ks.n_variants; ++k) minb[k] = c->ks.variant_minb[k];
    return LBM_OK;
}

int lbm_set_variant(lbm_ctx* c, int v) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!c->built) return fail(LBM_ERR_STATE, "grid not built");
    if (v < 0 || v >= c->ks.n_variants) return fail(LBM_ERR_ARG, "variant out of range");
    c->ks.step = c->ks.variant[v];
    c->variant = v;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return LBM_OK;
}

int lbm_mlp_set(lbm_ctx* c, const float* params, const double m[8], const double s[8]) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!params || !m || !s) return fail(LBM_ERR_ARG, "null argument");
    if (c->host_only) return fail(LBM_ERR_STATE, "host-only context");
    const int np = lbm_mlp_nparams();
    std::vector<float> h(params, params + np);
    // weight matrices rounded once (biases kept): [W1 192, b1 64, W2 4096, b2 64, W3 512, b3 8]
    const int w_ranges[3][2] = {{0, 192}, {256, 4352}, {4416, 4928}};
    for (auto& r : w_ranges)
        for (int k = r[0]; k < r[1]; ++k) h[k] = bf16_round_host(h[k]);
    CU(cudaSetDevice(c->device));
    if (!c->d_mlp && cudaMalloc(&c->d_mlp, np * sizeof(float)) != cudaSuccess) {
        c->d_mlp = nullptr;
        return fail(LBM_ERR_OOM, "network parameters");
    }
    CU(cudaMemcpy(c->d_mlp, h.data(), np * sizeof(float), cudaMemcpyHostToDevice));
    c->mlp_master.assign(params, params + np);
    for (int k = 0; k < 8; ++k) { c->mlp_m[k] = m[k]; c->mlp_s[k] = s[k]; }
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return LBM_OK;
}

int lbm_mlp_get(lbm_ctx* c, float* params, double m[8], double s[8]) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!params || !m || !s) return fail(LBM_ERR_ARG, "null argument");
    if (!c->d_mlp || c->mlp_master.empty()) return fail(LBM_ERR_STATE, "no network set");
    std::memcpy(params, c->mlp_master.data(), c->mlp_master.size() * sizeof(float));
    for (int k = 0; k < 8; ++k) { m[k] = c->mlp_m[k]; s[k] = c->mlp_s[k]; }
    return LBM_OK;
}

int lbm_mlp_train(lbm_ctx* c, const double* d_uT, const double* d_lambda, int64_t n, lbm_mlp_train_params* p) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!d_uT || !d_lambda || !p || n <= 0) return fail(LBM_ERR_ARG, "bad arguments");
    if (p->steps < 1 || p->batch < 1 || !(p->lr > 0) || p->lr_final < 0) return fail(LBM_ERR_ARG, "bad training parameters");
    if (c->host_only) return fail(LBM_ERR_STATE, "host-only context");
    if (c->model != LBM_COMP_NUMERICAL) return fail(LBM_ERR_UNSUPPORTED, "needs a numerical-equilibrium model");
    CU(cudaSetDevice(c->device));
    const int np = lbm_mlp_nparams();
    if (!c->d_mlp && cudaMalloc(&c->d_mlp, np * sizeof(float)) != cudaSuccess) {
        c->d_mlp = nullptr;
        return fail(LBM_ERR_OOM, "network parameters");
    }
    float* master = nullptr;
    CU(cudaMalloc(&master, np * sizeof(float)));
    double ms[16];
    const int r = mlp_train_device(d_uT, d_lambda, n, c->T0(), *p, master, c->d_mlp, ms, &p->final_loss, c->stream);
    if (r == LBM_OK) {
        c->mlp_master.resize(np);
        cudaMemcpy(c->mlp_master.data(), master, np * sizeof(float), cudaMemcpyDeviceToHost);
        for (int k = 0; k < 8; ++k) { c->mlp_m[k] = ms[k]; c->mlp_s[k] = ms[8 + k]; }
        if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    }
    cudaFree(master);
    return r;
}

int lbm_newton_batch(lbm_ctx* c, const double* d_uT, int64_t n, int guess, double* d_lambda, int* d_iters) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!d_uT || !d_lambda || !d_iters || n < 0) return fail(LBM_ERR_ARG, "bad arguments");
    if (c->host_only || !c->built) return fail(LBM_ERR_STATE, "grid not built on a device");
    if (c->model != LBM_COMP_NUMERICAL) return fail(LBM_ERR_UNSUPPORTED, "needs a numerical-equilibrium model");
    if (guess < LBM_GUESS_ZERO || guess > LBM_GUESS_MLP) return fail(LBM_ERR_ARG, "guess must be ZERO, POLY or MLP");
    if (guess == LBM_GUESS_MLP && !c->d_mlp) return fail(LBM_ERR_STATE, "no network set");
    CU(cudaSetDevice(c->device));
    StepArgs a;
    fill_args(c, a);
    ModelDev m = a.m;
    m.guess = guess;
    if (c->lattice == LBM_D2Q37) launch_newton_batch_d2q37(d_uT, n, m, d_lambda, d_iters, c->stream);
    else if (c->lattice == LBM_D2Q13) launch_newton_batch_d2q13(d_uT, n, m, d_lambda, d_iters, c->stream);
    else launch_newton_batch_d2q21(d_uT, n, m, d_lambda, d_iters, c->stream);
    CU(cudaGetLastError());
    return LBM_OK;
}

// ---------------------------------------------------------------- checkpoint
// File: magic, format version, a signature of the configuration (lattice, model, storage, block,
// levels, blocks and cell counts per level, a checksum of the cell types), the fine iteration
// counter, the device status and Newton counters, then per level the populations of both
// buffers (f, g) and the multipliers, as stored.
namespace {
constexpr uint64_t CKPT_MAGIC = 0x4C424D545245454BULL;   // "LBMTREEK"
constexpr uint32_t CKPT_VERSION = 1;

struct CkptHeader {
    uint64_t magic;
    uint32_t version, lattice, model, storage;
    int32_t block[3], n_levels;
    int64_t nb[8], ncell[8];
    uint64_t type_sum;
    int64_t t;
};

CkptHeader ckpt_header(const lbm_ctx* c) {
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = CKPT_MAGIC;
    h.version = CKPT_VERSION;
    h.lattice = (uint32_t)c->lattice;
    h.model = (uint32_t)c->model;
    h.storage = (uint32_t)c->storage;
    for (int d = 0; d < 3; ++d) h.block[d] = c->block[d];
    h.n_levels = c->L();
    uint64_t s = 1469598103934665603ULL;               // FNV-1a over the cell types
    for (int i = 0; i < c->L() && i < 8; ++i) {
        const BuiltLevel& lv = c->grid.levels[i];
        h.nb[i] = lv.nb;
        h.ncell[i] = lv.nb * c->grid.BS;
        for (uint8_t v : lv.type) s = (s ^ v) * 1099511628211ULL;
    }
    h.type_sum = s;
    h.t = c->t;
    return h;
}

// the device arrays of the state with their sizes in bytes
std::vector<std::pair<void*, size_t>> state_arrays(lbm_ctx* c) {
    std::vector<std::pair<void*, size_t>> v;
    const int Q = c->grid.lat.Q;
    const size_t es = c->storage == LBM_F64 ? 8 : c->storage == LBM_F32 ? 4 : 2;
    for (int i = 0; i < c->L(); ++i) {
        const int64_t ncell = c->grid.levels[i].nb * c->grid.BS;
        const size_t bytes = size_t(Q) * (ncell + c->grid.BS) * es;
        for (int k = 0; k < 2; ++k) {
            v.push_back({c->dl[i].f[k], bytes});
            if (c->dl[i].g[k]) v.push_back({c->dl[i].g[k], bytes});
        }
        if (c->dl[i].lam) v.push_back({c->dl[i].lam, size_t(2) * 8 * ncell * 8});
    }
    v.push_back({c->d_status, sizeof(int)});
    v.push_back({c->d_nstat, 19 * sizeof(unsigned long long)});
    return v;
}
}  // namespace

int lbm_save(lbm_ctx* c, const char* path) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!path) return fail(LBM_ERR_ARG, "null path");
    if (int r = ready(c)) return r;
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(LBM_ERR_ARG, std::string("cannot open ") + path);
    const CkptHeader h = ckpt_header(c);
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1;
    std::vector<char> buf;
    for (auto& [p, n] : state_arrays(c)) {
        if (!ok) break;
        buf.resize(n);
        if (cudaMemcpy(buf.data(), p, n, cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(fp);
            return fail(LBM_ERR_CUDA, "checkpoint read-back");
        }
        ok = std::fwrite(buf.data(), 1, n, fp) == n;
    }
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(LBM_ERR_ARG, std::string("write failed: ") + path);
}

int lbm_load(lbm_ctx* c, const char* path) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!path) return fail(LBM_ERR_ARG, "null path");
    if (!c->built || c->host_only) return fail(LBM_ERR_STATE, "build the same grid on a device first");
    CU(cudaSetDevice(c->device));
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(LBM_ERR_ARG, std::string("cannot open ") + path);
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    if (std::fread(&h, sizeof(h), 1, fp) != 1 || h.magic != CKPT_MAGIC || h.version != CKPT_VERSION) {
        std::fclose(fp);
        return fail(LBM_ERR_ARG, "not a checkpoint of this format");
    }
    CkptHeader mine = ckpt_header(c);
    mine.t = h.t;
    if (std::memcmp(&h, &mine, sizeof(h)) != 0) {
        std::fclose(fp);
        return fail(LBM_ERR_STATE, "checkpoint of another configuration or grid");
    }
    std::vector<char> buf;
    for (auto& [p, n] : state_arrays(c)) {
        buf.resize(n);
        if (std::fread(buf.data(), 1, n, fp) != n) {
            std::fclose(fp);
            return fail(LBM_ERR_ARG, "truncated checkpoint");
        }
        if (cudaMemcpy(p, buf.data(), n, cudaMemcpyHostToDevice) != cudaSuccess) {
            std::fclose(fp);
            return fail(LBM_ERR_CUDA, "checkpoint upload");
        }
    }
    std::fclose(fp);
    c->t = h.t;
    c->initialized = true;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return LBM_OK;
}

// ---------------------------------------------------------------- variant tuning
int lbm_autotune(lbm_ctx* c, int n_coarse, int* best_variant, float* ms_per_step) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (int r = ready(c)) return r;
    if (n_coarse < 1) return fail(LBM_ERR_ARG, "n_coarse must be positive");
    CU(cudaSetDevice(c->device));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    int best = c->variant;
    float best_ms = -1.0f;
    const int saved = c->variant;
    for (int v = 0; v < c->ks.n_variants; ++v) {
        lbm_set_variant(c, v);
        if (int r = lbm_step(c, 1)) return r;                 // warm-up (builds the graph)
        cudaEventRecord(e0, c->stream);
        if (int r = lbm_step(c, n_coarse)) return r;
        cudaEventRecord(e1, c->stream);
        CU(cudaEventSynchronize(e1));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)n_coarse;
        if (ms_per_step) ms_per_step[v] = ms;
        if (best_ms < 0 || ms < best_ms) { best_ms = ms; best = v; }
    }
    (void)saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lbm_set_variant(c, best);
    if (best_variant) *best_variant = best;
    return LBM_OK;
}

int lbm_use_graph(lbm_ctx* c, int on) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    c->use_graph = on != 0;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int64_t n_coarse) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (int r = ready(c)) return r;
    if (n_coarse < 0) return fail(LBM_ERR_ARG, "negative step count");
    const int64_t P = c->period();
    int64_t n = n_coarse * P;
    if (!c->use_graph) return launch_iterations(c, n);
    const int64_t span = 2 * P;
    while (n > 0 && c->t % span) {         // align to the captured span with plain launches
        if (int r = launch_iterations(c, 1)) return r;
        --n;
    }
    if (n >= span) {
        if (int r = build_graph(c)) return r;
        const int per = launches_per_span(c);
        for (; n >= span; n -= span) {
            CU(cudaGraphLaunch(c->gexec, c->stream));
            c->t += span;
            c->launches += per;
        }
    }
    return launch_iterations(c, n);
}

int lbm_sync(lbm_ctx* c) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (c->host_only || !c->built) return LBM_OK;
    CU(cudaStreamSynchronize(c->stream));
    int st = 0;
    CU(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) return fail(st, "device status " + std::to_string(st));
    return LBM_OK;
}

// readout of per-cell quantities (which: 0 moments rho, u(3), T; 1 f; 2 g; 3 lambda) into a
// device buffer in listing order, ncomp components of n values each
static int read_common(lbm_ctx* c, int which, int ncomp, double** d_out) {
    if (int r = ready(c)) return r;
    if (int r = ensure_slots(c)) return r;
    StepArgs a;
    current_args(c, a);
    const int BS = c->grid.BS;
    const int64_t n = (int64_t)c->h_type.size();
    int64_t maxcell = 0;
    for (int i = 0; i < c->L(); ++i) maxcell = std::max<int64_t>(maxcell, c->grid.levels[i].nb * BS);
    // scratch kept by the context between reads (grown on demand)
    const size_t need_lev = size_t(ncomp) * maxcell * 8, need_lst = size_t(ncomp) * n * 8;
    if (c->rd_lev_bytes < need_lev) {
        if (c->d_rd_lev) cudaFree(c->d_rd_lev);
        c->d_rd_lev = nullptr;
        c->rd_lev_bytes = 0;
        if (cudaMalloc(&c->d_rd_lev, need_lev) != cudaSuccess) { c->d_rd_lev = nullptr; return fail(LBM_ERR_OOM, "readout buffer"); }
        c->rd_lev_bytes = need_lev;
    }
    if (c->rd_lst_bytes < need_lst) {
        if (c->d_rd_lst) cudaFree(c->d_rd_lst);
        c->d_rd_lst = nullptr;
        c->rd_lst_bytes = 0;
        if (cudaMalloc(&c->d_rd_lst, need_lst) != cudaSuccess) { c->d_rd_lst = nullptr; return fail(LBM_ERR_OOM, "readout buffer"); }
        c->rd_lst_bytes = need_lst;
    }
    double* d = c->d_rd_lev;
    double* lst = c->d_rd_lst;
    for (int i = 0; i < c->L(); ++i) {
        const int64_t ncell = c->grid.levels[i].nb * BS;
        if (!ncell) continue;
        const int64_t f0 = c->level_first[i], cnt = c->level_first[i + 1] - f0;
        cudaMemsetAsync(d, 0, size_t(ncomp) * ncell * 8, c->stream);
        c->ks.read(a, i, which, d, c->stream);
        launch_gather(c->d_slot + f0, cnt, d, ncell, ncomp, lst + f0, n, c->stream);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("readout: ") + cudaGetErrorString(e));
    *d_out = lst;
    return LBM_OK;
}

int lbm_read_moments(lbm_ctx* c, double* rho, double* u, double* T) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!rho || !u) return fail(LBM_ERR_ARG, "null output");
    double* lst = nullptr;
    if (int r = read_common(c, 0, 5, &lst)) return r;
    const int64_t n = (int64_t)c->h_type.size();
    cudaError_t e = cudaMemcpy(rho, lst, size_t(n) * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(u, lst + n, size_t(c->dim) * n * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && T) e = cudaMemcpy(T, lst + 4 * n, size_t(n) * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("readout copy: ") + cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_read_populations(lbm_ctx* c, int which, double* out) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!out || which < 0 || which > 2) return fail(LBM_ERR_ARG, "bad arguments");
    if (which == 1 && !c->comp()) return fail(LBM_ERR_ARG, "model has no g populations");
    if (which == 2 && c->model != LBM_COMP_NUMERICAL) return fail(LBM_ERR_ARG, "model has no multipliers");
    const int ncomp = which == 2 ? 8 : c->grid.lat.Q;
    double* lst = nullptr;
    if (int r = read_common(c, which + 1, ncomp, &lst)) return r;
    const int64_t n = (int64_t)c->h_type.size();
    cudaError_t e = cudaMemcpy(out, lst, size_t(ncomp) * n * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("readout copy: ") + cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_conserved(lbm_ctx* c, double out[5]) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!out) return fail(LBM_ERR_ARG, "null output");
    if (int r = ready(c)) return r;
    if (c->t % c->period()) return fail(LBM_ERR_STATE, "not at a coarse synchronisation instant");
    StepArgs a;
    const int64_t nb = current_args(c, a);
    c->ks.ledger(a, nb, c->d_partial, c->d_out5, c->stream);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(out, c->d_out5, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 5; ++k)
        if (!std::isfinite(out[k])) return fail(LBM_ERR_NONFINITE, "the state holds NaN or Inf (conserved totals not finite)");
    return LBM_OK;
}

int lbm_stats(lbm_ctx* c, lbm_stats_t* s) {
    if (check_ctx(c)) return LBM_ERR_ARG;
    if (!s) return fail(LBM_ERR_ARG, "null output");
    std::memset(s, 0, sizeof(*s));
    if (!c->built) return fail(LBM_ERR_STATE, "grid not built");
    s->n_levels = c->L();
    for (int d = 0; d < 3; ++d) s->block[d] = c->block[d];
    for (int i = 0; i < c->L() && i < 8; ++i) {
        const BuiltLevel& lv = c->grid.levels[i];
        s->n_blocks[i] = lv.nb;
        for (int64_t b = 0; b < lv.nb; ++b) s->n_general_blocks[i] += lv.bflag[b] ? 0 : 1;
        s->n_cells[i] = lv.count[1] + lv.count[2] + lv.count[3] + lv.count[4] + lv.count[5];
        const int64_t live = lv.count[1] + lv.count[2] + lv.count[3] + lv.count[4];
        s->cell_updates += live << (c->L() - 1 - i);
    }
    s->n_eq = c->grid.n_eq;
    s->fine_iterations = c->t + c->t_offset;
    s->kernel_launches = c->launches;
    s->device_bytes = c->dev_bytes;
    if (!c->host_only && c->d_nstat) {
        unsigned long long h[19];
        CU(cudaStreamSynchronize(c->stream));
        CU(cudaMemcpy(h, c->d_nstat, sizeof(h), cudaMemcpyDeviceToHost));
        s->newton_iter_sum = (int64_t)h[0];
        s->newton_updates = (int64_t)h[1];
        s->newton_nonconverged = (int64_t)h[2];
        for (int k = 0; k < 16; ++k) s->newton_hist[k] = (int64_t)h[3 + k];
    }
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batched cases
// Cases that share lattice, model, storage, block shape and step variant form a group; every
// fine iteration launches each group's FAST and general kernels once over the active blocks of
// all its cases.  The per-case iteration arguments of a span of 2^L fine iterations (L the
// largest level count) sit in a device table; the span is captured as a CUDA graph.
struct lbm_batch {
    struct Group {
        KernelSet ks;
        int variant = 0;
        std::vector<int> cases;                 // indices into lbm_batch::cases
        StepArgs* d_args = nullptr;             // span x n
        long long* d_off = nullptr;             // span x 2 x (n + 1)
        std::vector<long long> nf, ng;          // per iteration of the span
    };
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;                // general kernels, forked and joined per iteration
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<lbm_ctx*> cases;
    std::vector<int64_t> t0;                    // case times when the tables were built
    std::vector<Group> groups;
    int64_t span = 1, tb = 0;
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    int64_t launches = 0;

    void release_streams() {
        if (side) { cudaStreamSynchronize(side); cudaStreamDestroy(side); side = nullptr; }
        if (ev_fork) { cudaEventDestroy(ev_fork); ev_fork = nullptr; }
        if (ev_join) { cudaEventDestroy(ev_join); ev_join = nullptr; }
        if (own_stream && stream) { cudaStreamDestroy(stream); stream = nullptr; }
    }
    void free_tables() {
        if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
        for (auto& g : groups) {
            if (g.d_args) cudaFree(g.d_args);
            if (g.d_off) cudaFree(g.d_off);
            g.d_args = nullptr;
            g.d_off = nullptr;
        }
    }
};

namespace {

int batch_tables(lbm_batch* b) {
    b->free_tables();
    b->span = 1;
    for (lbm_ctx* c : b->cases) b->span = std::max(b->span, 2 * c->period());
    b->t0.resize(b->cases.size());
    for (size_t k = 0; k < b->cases.size(); ++k) b->t0[k] = b->cases[k]->t;
    b->tb = 0;
    for (auto& g : b->groups) {
        const int n = (int)g.cases.size();
        std::vector<StepArgs> args(size_t(b->span) * n);
        std::vector<long long> off(size_t(b->span) * 2 * (n + 1));
        g.nf.assign(b->span, 0);
        g.ng.assign(b->span, 0);
        for (int64_t j = 0; j < b->span; ++j) {
            long long* of = &off[size_t(j) * 2 * (n + 1)];
            long long* og = of + (n + 1);
            of[0] = og[0] = 0;
            for (int k = 0; k < n; ++k) {
                lbm_ctx* c = b->cases[g.cases[k]];
                StepArgs& a = args[size_t(j) * n + k];
                iteration_args(c, c->t + j, a);
                of[k + 1] = of[k] + a.list_off[0][a.n_active];
                og[k + 1] = og[k] + a.list_off[1][a.n_active];
            }
            g.nf[j] = of[n];
            g.ng[j] = og[n];
        }
        CU(cudaMalloc(&g.d_args, args.size() * sizeof(StepArgs)));
        CU(cudaMalloc(&g.d_off, off.size() * sizeof(long long)));
        CU(cudaMemcpy(g.d_args, args.data(), args.size() * sizeof(StepArgs), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(g.d_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice));
    }
    return LBM_OK;
}

// one fine iteration of every case (table row j); general kernels on the side stream
void batch_iteration(lbm_batch* b, int64_t j) {
    cudaEventRecord(b->ev_fork, b->stream);
    cudaStreamWaitEvent(b->side, b->ev_fork, 0);
    for (auto& g : b->groups) {
        const int n = (int)g.cases.size();
        const long long* of = g.d_off + size_t(j) * 2 * (n + 1);
        g.ks.batch[g.variant](g.d_args + size_t(j) * n, of, of + (n + 1), n, g.nf[j], g.ng[j], b->stream, b->side);
        b->launches += (g.nf[j] > 0) + (g.ng[j] > 0);
    }
    cudaEventRecord(b->ev_join, b->side);
    cudaStreamWaitEvent(b->stream, b->ev_join, 0);
}

int batch_graph(lbm_batch* b) {
    if (b->gexec) return LBM_OK;
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t saved = b->launches;
    for (int64_t j = 0; j < b->span; ++j) batch_iteration(b, j);
    b->launches = saved;
    if (cudaGetLastError() != cudaSuccess) {
        cudaGraph_t g2 = nullptr;
        cudaStreamEndCapture(b->stream, &g2);
        if (g2) cudaGraphDestroy(g2);
        return fail(LBM_ERR_CUDA, "launch during graph capture failed");
    }
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch** out, lbm_ctx* const* cases, int n, void* stream) {
    if (!out) return fail(LBM_ERR_ARG, "out is null");
    *out = nullptr;
    if (!cases || n <= 0) return fail(LBM_ERR_ARG, "no cases");
    for (int k = 0; k < n; ++k) {
        if (check_ctx(cases[k])) return LBM_ERR_ARG;
        if (int r = ready(cases[k])) return r;
        if (cases[k]->device != cases[0]->device) return fail(LBM_ERR_ARG, "cases on different devices");
        if (cases[k]->streaming != LBM_STREAM_AB) return fail(LBM_ERR_UNSUPPORTED, "batched cases use two-buffer streaming");
        for (int j = 0; j < k; ++j)
            if (cases[j] == cases[k]) return fail(LBM_ERR_ARG, "a case is listed twice");
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return fail(LBM_ERR_OOM, "batch allocation");
    b->device = cases[0]->device;
    b->cases.assign(cases, cases + n);
    for (int k = 0; k < n; ++k) {
        lbm_ctx* c = cases[k];
        if (!c->ks.batch[c->variant]) {
            delete b;
            return fail(LBM_ERR_UNSUPPORTED, "no batched kernels for this lattice (D2Q9 and D2Q37 have them)");
        }
        bool placed = false;
        for (auto& g : b->groups) {
            lbm_ctx* h = b->cases[g.cases[0]];
            if (h->lattice == c->lattice && h->model == c->model && h->storage == c->storage &&
                h->block[0] == c->block[0] && h->block[1] == c->block[1] && h->block[2] == c->block[2] &&
                h->variant == c->variant) {
                g.cases.push_back(k);
                placed = true;
                break;
            }
        }
        if (!placed) {
            lbm_batch::Group g;
            g.ks = c->ks;
            g.variant = c->variant;
            g.cases.push_back(k);
            b->groups.push_back(std::move(g));
        }
    }
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) {
        b->stream = (cudaStream_t)stream;
        if (!b->stream) {
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
            b->own_stream = e == cudaSuccess;
        }
    }
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        b->release_streams();
        delete b;
        return fail(LBM_ERR_CUDA, std::string("batch stream: ") + cudaGetErrorString(e));
    }
    // the cases' own streams may hold queued work
    for (lbm_ctx* c : b->cases) cudaStreamSynchronize(c->stream);
    if (int r = batch_tables(b)) {
        b->free_tables();
        b->release_streams();
        delete b;
        return r;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    cudaSetDevice(b->device);
    b->free_tables();
    b->release_streams();
    delete b;
    return LBM_OK;
}

int lbm_batch_use_graph(lbm_batch* b, int on) {
    if (!b) return fail(LBM_ERR_ARG, "null batch");
    b->use_graph = on != 0;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t n_fine) {
    if (!b) return fail(LBM_ERR_ARG, "null batch");
    if (n_fine < 0) return fail(LBM_ERR_ARG, "negative step count");
    CU(cudaSetDevice(b->device));
    // a case stepped on its own since the tables were built: rebuild them at its new time
    bool moved = false;
    for (size_t k = 0; k < b->cases.size(); ++k) {
        lbm_ctx* c = b->cases[k];
        if (int r = ready(c)) return r;
        if (c->t != b->t0[k] + b->tb) moved = true;
    }
    if (moved) {
        for (lbm_ctx* c : b->cases) cudaStreamSynchronize(c->stream);
        if (int r = batch_tables(b)) return r;
    }
    int64_t n = n_fine;
    while (n > 0) {
        const int64_t j = b->tb % b->span;
        if (b->use_graph && j == 0 && n >= b->span) {
            if (int r = batch_graph(b)) return r;
            CU(cudaGraphLaunch(b->gexec, b->stream));
            for (auto& g : b->groups)
                for (int64_t i = 0; i < b->span; ++i) b->launches += (g.nf[i] > 0) + (g.ng[i] > 0);
            b->tb += b->span;
            n -= b->span;
            for (lbm_ctx* c : b->cases) c->t += b->span;
            continue;
        }
        batch_iteration(b, j);
        b->tb++;
        n--;
        for (lbm_ctx* c : b->cases) c->t++;
    }
    CU(cudaGetLastError());
    // later work on a case's own stream runs after the batch
    cudaEvent_t ev;
    CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CU(cudaEventRecord(ev, b->stream));
    for (lbm_ctx* c : b->cases) cudaStreamWaitEvent(c->stream, ev, 0);
    cudaEventDestroy(ev);
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch* b) {
    if (!b) return fail(LBM_ERR_ARG, "null batch");
    CU(cudaSetDevice(b->device));
    CU(cudaStreamSynchronize(b->stream));
    for (lbm_ctx* c : b->cases)
        if (int r = lbm_sync(c)) return r;
    return LBM_OK;
}

int lbm_batch_info(lbm_batch* b, int* n_groups, int64_t* launches, int64_t* span) {
    if (!b) return fail(LBM_ERR_ARG, "null batch");
    if (n_groups) *n_groups = (int)b->groups.size();
    if (launches) *launches = b->launches;
    if (span) *span = b->span;
    return LBM_OK;
}

}  // extern "C"
