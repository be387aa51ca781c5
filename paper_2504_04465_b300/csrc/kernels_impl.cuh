// Kernel templates of the CUDA path: fused collide-and-stream over all active levels,
// initialisation, moment/population readout and the FP64 conservation ledger.  Each lattice's
// translation unit (k_d2q9.cu, k_d3q27.cu, k_d2q37.cu, k_d2q21.cu) defines its model policy and
// instantiates them.
//
// One launch per fine iteration covers every level active at that iteration (Sec. 4.5 of
// arXiv 2504.04465 runs them one after the other; the paper's future work proposes loading the
// GPU with all active levels at once).  This is race-free in the pull form: level i reads its
// own buffer rd_i and writes rd_i ^ 1; the coupling of level i with i-1 (Sec. 3.2) is fused into
// level i's coarse-ghost cells, which read level i-1's buffer rd_{i-1} (coalescence) and write the
// fine-ghost slots of rd_{i-1} ^ 1 (explosion); level i-1 skips its fine ghosts at that iteration.
//
// Model policy M: D, Q, DEV (values are deviations f - w rho_ref), HAS_G, HAS_LAM, RR,
// cx/cy/cz(q), w(q); compressible models also
//   template <int ST> static void feq(m, rho, ux, uy, T, lam, feq, iters, conv)
//   static void init_guess(ux, uy, T, lam)
#pragma once
#include <type_traits>
#include <utility>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"
#include "models.cuh"
#include "models_comp.cuh"

namespace lbm {

// Weakly compressible models on lattices that are not tensor products of D1Q3 (D2Q21) carry
// their own equilibrium and collision (HERMITE_WEAK); the others use the separable forms.
template <class M, class = void> struct hermite_weak : std::false_type {};
template <class M>
struct hermite_weak<M, std::void_t<decltype(M::HERMITE_WEAK)>> : std::bool_constant<M::HERMITE_WEAK> {};


// collision variant of a weakly compressible tensor-product model (WV_*; 0 where not declared)
template <class M, class = void> struct weak_var : std::integral_constant<int, 0> {};
template <class M>
struct weak_var<M, std::void_t<decltype(M::VAR)>> : std::integral_constant<int, M::VAR> {};

// models compiled with the AA-pattern kernels (M::AA)
template <class M, class = void> struct aa_capable : std::false_type {};
template <class M>
struct aa_capable<M, std::void_t<decltype(M::AA)>> : std::bool_constant<M::AA> {};

enum Mode { MODE_STEP = 0, MODE_READ = 1, MODE_LEDGER = 2 };

// largest |xi_a| of the lattice (its reach)
template <class M>
__host__ __device__ constexpr int lattice_reach() {
    int r = 0;
    for (int q = 0; q < M::Q; ++q) {
        const int a = M::cx(q) < 0 ? -M::cx(q) : M::cx(q), b = M::cy(q) < 0 ? -M::cy(q) : M::cy(q),
                  c = M::cz(q) < 0 ? -M::cz(q) : M::cz(q);
        r = a > r ? a : r;
        r = b > r ? b : r;
        r = c > r ? c : r;
    }
    return r;
}

// Concave corners of the finer region: over one coarse step a fine ghost only streams, so the
// population xi of child ch at the coalescence left ch - 2 xi through ch - xi.  True when that
// history leaves the finer level (ch - xi is no cell of it, or is a fine ghost and ch - 2 xi is
// none): the packet came from the coarse side and the coarse ghost's own streamed population
// stands in for it.  Two steps of the lattice reach stay within the neighbouring blocks.
template <class M, int BX, int BY, int BZ>
__device__ __forceinline__ bool history_leaves(const LevelDev& F, long long ch, int cx, int cy, int cz) {
    static_assert(2 * lattice_reach<M>() <= BX && 2 * lattice_reach<M>() <= BY &&
                      (M::D == 2 || 2 * lattice_reach<M>() <= BZ),
                  "two lattice steps must stay within the neighbouring blocks");
    const long long s1 = src_cell_g<BX, BY, BZ>(F.nbr, ch, cx, cy, cz);
    if (s1 < 0) return true;
    const int t1 = F.type[s1];
    if (t1 == C_ABSENT) return true;
    if (t1 != C_FGHOST) return false;
    const long long s2 = src_cell_g<BX, BY, BZ>(F.nbr, ch, 2 * cx, 2 * cy, 2 * cz);
    return s2 < 0 || F.type[s2] == C_ABSENT;
}

template <class M, int ST>
struct Cell {
    using T = typename Store<ST>::T;
    T f[M::Q];
    T g[M::HAS_G ? M::Q : 1];
    double lam[M::HAS_LAM ? 8 : 1];
};

// reference values w_q rho_ref (f) and w_q rho_ref (2 Cv - D) T0 (g) of the deviation formats, and
// their reciprocals; in FP32 from single-precision weights, so that no FP64 operation or
// division is left in the per-population path
template <class M, int ST>
__device__ __forceinline__ typename Store<ST>::T ref_f(const ModelDev& m, int q) {
    using T = typename Store<ST>::T;
    if constexpr (sizeof(T) == 4) return M::wf(q) * m.rho_ref_f;
    else return T(M::w(q) * m.rho_ref);
}
template <class M, int ST>
__device__ __forceinline__ typename Store<ST>::T inv_ref_f(const ModelDev& m, int q) {
    using T = typename Store<ST>::T;
    if constexpr (sizeof(T) == 4) return M::inv_wf(q) * m.inv_rho_ref_f;
    else return T(1.0 / (M::w(q) * m.rho_ref));
}
template <class M, int ST>
__device__ __forceinline__ typename Store<ST>::T ref_g(const ModelDev& m, int q) {
    using T = typename Store<ST>::T;
    if constexpr (sizeof(T) == 4) return M::wf(q) * m.gref_f;
    else return T(M::w(q) * m.rho_ref * (2.0 * m.Cv - M::D) * m.T0);
}
template <class M, int ST>
__device__ __forceinline__ typename Store<ST>::T inv_ref_g(const ModelDev& m, int q) {
    using T = typename Store<ST>::T;
    if constexpr (sizeof(T) == 4) return M::inv_wf(q) * m.inv_gref_f;
    else return T(1.0 / (M::w(q) * m.rho_ref * (2.0 * m.Cv - M::D) * m.T0));
}

template <class M, int ST, int BS>
__device__ __forceinline__ void load_pop(const LevelDev& L, int buf, long long src, int q, const ModelDev& m,
                                         typename Store<ST>::T& fo, typename Store<ST>::T& go) {
    using T = typename Store<ST>::T;
    if (src < 0) {                                       // no source: a zero population
        fo = M::DEV ? -ref_f<M, ST>(m, q) : T(0);
        go = T(0);
        return;
    }
    const long long i = pidx<BS, M::Q>(src, q);
    fo = Store<ST>::template load<M::DEV>(L.f[buf], i, ref_f<M, ST>(m, q));
    if constexpr (M::HAS_G) go = Store<ST>::template load<false>(L.g[buf], i, ref_g<M, ST>(m, q));
    else go = T(0);
}

template <class M, int ST, int BS>
__device__ __forceinline__ void store_pop(const LevelDev& L, int buf, long long cell, int q, const ModelDev& m,
                                          typename Store<ST>::T fv, typename Store<ST>::T gv) {
    const long long i = pidx<BS, M::Q>(cell, q);
    Store<ST>::template store<M::DEV>(L.f[buf], i, fv, inv_ref_f<M, ST>(m, q));
    if constexpr (M::HAS_G) Store<ST>::template store<false>(L.g[buf], i, gv, inv_ref_g<M, ST>(m, q));
}

// macroscopic moments (rho, u, T) of f, g (T from Eq. polyTemp)
template <class M, int ST>
__device__ __forceinline__ void moments(const ModelDev& m, const Cell<M, ST>& c, typename Store<ST>::T& rho,
                                        typename Store<ST>::T* u, typename Store<ST>::T& Tt) {
    using T = typename Store<ST>::T;
    T r = M::DEV ? (sizeof(T) == 4 ? T(m.rho_ref_f) : T(m.rho_ref)) : T(0), jx = 0, jy = 0, jz = 0, e2 = 0, gs = 0;
#pragma unroll
    for (int q = 0; q < M::Q; ++q) {
        const T v = c.f[q];
        r += v;
        if (M::cx(q)) jx += T(M::cx(q)) * v;
        if (M::cy(q)) jy += T(M::cy(q)) * v;
        if (M::cz(q)) jz += T(M::cz(q)) * v;
        if constexpr (M::HAS_G) {
            e2 += T(M::cx(q) * M::cx(q) + M::cy(q) * M::cy(q)) * v;
            gs += c.g[q];
        }
    }
    rho = r;
    u[0] = jx / r;
    u[1] = jy / r;
    u[2] = jz / r;
    Tt = T(0);
    if constexpr (M::HAS_G) Tt = (e2 + gs - r * (u[0] * u[0] + u[1] * u[1])) / (T(2) * r * T(m.Cv));
}

// Ladd's moving-wall term of link q of cell l of block b (Appendix A.3): when the pull source
// leaves the domain through wall faces only, 2 w_q (xi_q . rho_w u_w) / c_s^2 with rho_w u_w the
// mean over the wall faces crossed (periodic axes wrap and are not crossings); 0 otherwise (a
// link blocked by a solid).  Weakly compressible models (c_s^2 = m.cs2).
template <class M, int BX, int BY, int BZ>
__device__ __forceinline__ double wall_term(const ModelDev& m, const LevelDev& L, long long b, int l, int q) {
    const int lc[3] = {L.bxyz[3 * b] * BX + l % BX, L.bxyz[3 * b + 1] * BY + (l / BX) % BY,
                       L.bxyz[3 * b + 2] * BZ + l / (BX * BY)};
    const int xi[3] = {M::cx(q), M::cy(q), M::cz(q)};
    double mom[3] = {0.0, 0.0, 0.0};
    int walls = 0;
#pragma unroll
    for (int d = 0; d < M::D; ++d) {
        const int s = lc[d] - xi[d];
        const int f = s < 0 ? 2 * d : (s >= L.shape[d] ? 2 * d + 1 : -1);
        if (f < 0 || m.faces[f].kind == LBM_PERIODIC) continue;
        if (m.faces[f].kind != LBM_WALL) return 0.0;
        ++walls;
#pragma unroll
        for (int k = 0; k < 3; ++k) mom[k] += m.faces[f].rho * m.faces[f].u[k];
    }
    if (!walls) return 0.0;
    const double dot = double(xi[0]) * mom[0] + double(xi[1]) * mom[1] + double(xi[2]) * mom[2];
    return 2.0 * M::w(q) * dot / (double(walls) * m.cs2);
}

// ------------------------------------------------------------------ state assembly
// Pre-collision state of the cell (level lev, block b, local l) at the current iteration:
//   FLUID : pull gather, bounce-back on blocked links
//   CGHOST: pull gather; in STEP/LEDGER modes the unknown populations are the mean of the
//           children's streamed populations (Eq. coalescence; at a concave corner a child whose
//           history left the finer level counts with the ghost's own streamed population) and
//           lambda the children's mean
//   FGHOST: pull gather (pure streaming), lambda carried
//   BC    : Neumann copies the partner's gathered state (and lambda); Dirichlet sets the
//           equilibrium of (rho_bc or the partner's rho, u_bc, T_bc)
template <class M, int ST, int BX, int BY, int BZ, int MODE>
__device__ __forceinline__ void assemble(const StepArgs& a, int lev, long long b, int l, int type, bool simple,
                                         const int* nbr_s, Cell<M, ST>& c, int* conv_out,
                                         const typename Store<ST>::T* coal_pre = nullptr) {
    using T = typename Store<ST>::T;
    constexpr int BS = BX * BY * BZ;
    const LevelDev& L = a.lv[lev];
    const int rd = a.rd[lev];
    const long long cell = b * BS + l;
    const int lx = l % BX, ly = (l / BX) % BY, lz = l / (BX * BY);
    *conv_out = 1;
    if (a.aa_l1 && type == C_FLUID) {
        // AA streaming, layout L1: the cell's own slot qbar holds f_q (bounces already in place)
#pragma unroll
        for (int q = 0; q < M::Q; ++q) {
            T gv = T(0);
            load_pop<M, ST, BX * BY * BZ>(L, rd, cell, M::Q - 1 - q, a.m, c.f[q], gv);
            if constexpr (M::HAS_G) c.g[q] = gv;
        }
        if constexpr (M::HAS_LAM) {
#pragma unroll
            for (int i = 0; i < 8; ++i) c.lam[i] = L.lam[((long long)rd * 8 + i) * L.ncell + cell];
        }
        return;
    }
    if (type != C_BC) {
        unsigned long long bmask = 0ull, umask = 0ull;
        long long child = -1;
        bool corner = false;    // a coarse ghost at a concave corner of the finer region
        bool walls = false;     // a fluid cell with links bounced at wall faces
        if (!simple && type != C_FGHOST) {
            const int r = L.rec_id[cell];
            if (r >= 0) {
                const CellRecDev rec = L.recs[r];
                if (type == C_FLUID) {
                    bmask = rec.mask;
                    walls = (rec.b & 2) != 0;
                } else {
                    umask = rec.mask;
                    child = rec.a;
                    corner = (rec.b & 1) != 0;
                }
            }
        }
        const bool coal = (type == C_CGHOST) && (MODE != MODE_READ);
#pragma unroll
        for (int q = 0; q < M::Q; ++q) {
            T gv = T(0);
            if (bmask & (1ull << q)) {
                load_pop<M, ST, BX * BY * BZ>(L, rd, cell, M::Q - 1 - q, a.m, c.f[q], gv);      // f_q(x) = f*_qbar(x)
                if constexpr (!M::HAS_G) {
                    if (walls) c.f[q] += T(wall_term<M, BX, BY, BZ>(a.m, L, b, l, q));
                }
            } else if (!(coal && (umask & (1ull << q))) || corner) {
                // (a corner ghost keeps its own streamed unknowns: they stand in for the
                // children whose history left the finer level)
                const long long s = src_cell<BX, BY, BZ>(nbr_s, b, lx, ly, lz, M::cx(q), M::cy(q), M::cz(q));
                load_pop<M, ST, BX * BY * BZ>(L, rd, s, q, a.m, c.f[q], gv);
            }
            if constexpr (M::HAS_G) c.g[q] = gv;
        }
        if (coal && coal_pre) {
            // coalesced values computed by the whole block beforehand ([q][cell] in shared memory)
#pragma unroll
            for (int q = 0; q < M::Q; ++q)
                if (umask & (1ull << q)) c.f[q] = coal_pre[q * BS + l];
        } else if (coal) {
            // coalescence: one population at a time (set bits of the unknown mask), its 2^D
            // children's streamed values loaded together and summed in child order
            const LevelDev& F = a.lv[lev - 1];
            const int rdf = a.rd[lev - 1];
            constexpr int NK = (M::D == 3) ? 8 : 4;
            unsigned long long um = umask;
#pragma unroll 1
            while (um) {
                const int q = __ffsll((long long)um) - 1;
                um &= um - 1;
                int cx = 0, cy = 0, cz = 0;
#pragma unroll
                for (int qq = 0; qq < M::Q; ++qq)
                    if (qq == q) { cx = M::cx(qq); cy = M::cy(qq); cz = M::cz(qq); }
                T own_f = T(0), own_g = T(0);
#pragma unroll
                for (int qq = 0; qq < M::Q; ++qq) {
                    if (qq == q) {
                        own_f = c.f[qq];
                        if constexpr (M::HAS_G) own_g = c.g[qq];
                    }
                }
                T vf[NK], vg[NK];
#pragma unroll
                for (int k = 0; k < NK; ++k) {
                    const long long ch = child + (k & 1) + ((k >> 1) & 1) * BX + ((k >> 2) & 1) * BX * BY;
                    if (corner && history_leaves<M, BX, BY, BZ>(F, ch, cx, cy, cz)) {
                        vf[k] = own_f;
                        vg[k] = own_g;
                        continue;
                    }
                    const long long s = src_cell_g<BX, BY, BZ>(F.nbr, ch, cx, cy, cz);
                    load_pop<M, ST, BX * BY * BZ>(F, rdf, s, q, a.m, vf[k], vg[k]);
                }
                T sf = 0, sg = 0;
#pragma unroll
                for (int k = 0; k < NK; ++k) {
                    sf += vf[k];
                    sg += vg[k];
                }
                sf = sf / T(NK);
                sg = sg / T(NK);
#pragma unroll
                for (int qq = 0; qq < M::Q; ++qq) {
                    if (qq == q) {
                        c.f[qq] = sf;
                        if constexpr (M::HAS_G) c.g[qq] = sg;
                    }
                }
            }
        }
        if constexpr (M::HAS_LAM) {
            if (coal) {
                const LevelDev& F = a.lv[lev - 1];
                const int rdf = a.rd[lev - 1];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    double s = 0.0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const long long ch = child + (k & 1) + ((k >> 1) & 1) * BX;
                        s += F.lam[((long long)rdf * 8 + i) * F.ncell + ch];
                    }
                    c.lam[i] = s / 4.0;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) c.lam[i] = L.lam[((long long)rd * 8 + i) * L.ncell + cell];
            }
        }
        return;
    }
    // boundary layer cell
    const CellRecDev rec = L.recs[L.rec_id[cell]];
    const long long P = rec.a;
    const int kind = rec.b & 15, face = rec.b >> 4;
#pragma unroll
    for (int q = 0; q < M::Q; ++q) {
        const long long s = src_cell_g<BX, BY, BZ>(L.nbr, P, M::cx(q), M::cy(q), M::cz(q));
        T gv;
        load_pop<M, ST, BX * BY * BZ>(L, rd, s, q, a.m, c.f[q], gv);
        if constexpr (M::HAS_G) c.g[q] = gv;
    }
    if constexpr (M::HAS_LAM) {
        const long long src = (kind == 3) ? P : cell;
#pragma unroll
        for (int i = 0; i < 8; ++i) c.lam[i] = L.lam[((long long)rd * 8 + i) * L.ncell + src];
    }
    if (kind == 3) return;                                     // Neumann
    const FaceDev& fd = a.m.faces[face];
    T rho = T(fd.rho);
    if (kind == 2) {                                           // extrapolated density
        T r = 0;
#pragma unroll
        for (int q = 0; q < M::Q; ++q) r += c.f[q];
        rho = M::DEV ? r + T(a.m.rho_ref) : r;
    }
    if constexpr (!M::HAS_G) {
        if constexpr (hermite_weak<M>::value) M::template feq_dev<T>(rho, T(fd.u[0]), T(fd.u[1]), T(a.m.rho_ref), c.f);
        else weak_feq_dev<M::D, T>(rho, T(fd.u[0]), T(fd.u[1]), T(fd.u[2]), T(a.m.rho_ref), c.f);
    } else {
        int it = 0, conv = 1;
        M::template feq<ST>(a.m, rho, T(fd.u[0]), T(fd.u[1]), T(fd.T), c.lam, c.f, &it, &conv);
        const T gfac = T((2.0 * a.m.Cv - M::D) * fd.T);
#pragma unroll
        for (int q = 0; q < M::Q; ++q) c.g[q] = gfac * c.f[q];
        *conv_out = conv;
    }
}

// ------------------------------------------------------------------ collision
// REL: write the binary16 storage value f*/(w rho_ref) - 1 (weakly compressible RR, F16DEV)
template <class M, int ST, bool REL = false>
__device__ __forceinline__ int collide(const ModelDev& m, const LevelDev& L, Cell<M, ST>& c, int* conv) {
    using T = typename Store<ST>::T;
    *conv = 1;
    const double tau = L.tau;
    if constexpr (!M::HAS_G) {
        if constexpr (hermite_weak<M>::value) {
            if constexpr (sizeof(T) == 4) M::template collide<T>(c.f, L.omega_f, m.rho_ref_f);
            else M::template collide<T>(c.f, T(L.omega), T(m.rho_ref));
        } else if constexpr (REL) weak_collide<M::D, true, T, true>(c.f, L.omega_f, m.rho_ref_f, m.inv_rho_ref_f);
        else if constexpr (sizeof(T) == 4)
            weak_collide<M::D, M::RR, T, false, weak_var<M>::value>(c.f, L.omega_f, m.rho_ref_f, T(1), L.omega_m_f);
        else weak_collide<M::D, M::RR, T, false, weak_var<M>::value>(c.f, T(L.omega), T(m.rho_ref), T(1), T(L.omega_m));
        return 0;
    } else {
        T rho, u[3], Tt;
        moments<M, ST>(m, c, rho, u, Tt);
        T feq[M::Q];
        int it = 0;
        M::template feq<ST>(m, rho, u[0], u[1], Tt, c.lam, feq, &it, conv);
        T tau_eff = T(tau);
        if (m.sensor_on) {
            T eps = 0;
            const T tiny = (sizeof(T) == 8) ? T(1e-300) : T(1e-30);
#pragma unroll
            for (int q = 0; q < M::Q; ++q)
                if (feq[q] > tiny) eps += sensor_ratio(r_fabs(c.f[q] - feq[q]), feq[q]);
            eps /= T(M::Q);
            tau_eff = T(tau) * sensor_alpha<T>(eps, T(tau), T(m.sensor_A));
        }
        const T gfac = T(2.0 * m.Cv - M::D) * Tt;
        const T om = T(1) / tau_eff;
#pragma unroll
        for (int q = 0; q < M::Q; ++q) {
            c.f[q] -= (c.f[q] - feq[q]) * om;
            c.g[q] -= (c.g[q] - gfac * feq[q]) * om;
        }
        return it;
    }
}

__device__ __forceinline__ int find_level(const StepArgs& a, long long bid, long long* b) {
    int k = 0;
    while (k + 1 < a.n_active && bid >= a.block_off[k + 1]) ++k;
    *b = bid - a.block_off[k];
    return a.active[k];
}

// ------------------------------------------------------------------ step kernels
// FAST = true runs the simple blocks (branch-free gather, no records), FAST = false the others
// (coarse and fine ghosts, boundary layers, cells next to solids).  Both read buffer rd and write
// rd ^ 1 of disjoint cells, so the two launches of an iteration are independent.
__device__ __forceinline__ int find_level_list(const StepArgs& a, int list, long long bid, long long* i) {
    int k = 0;
    while (k + 1 < a.n_active && bid >= a.list_off[list][k + 1]) ++k;
    *i = bid - a.list_off[list][k];
    return a.active[k];
}

// Pull-source term of one axis for local coordinate lc and velocity component c: the source
// lc - c wrapped into the block (neighbour digit o + 1 in {0, 1, 2}, scaled by DIG) and its
// local offset scaled by STRIDE, packed as (digit << 20) | offset.
template <int B, int STRIDE, int DIG>
__device__ __forceinline__ unsigned axis_term(int lc, int c) {
    int s = lc - c;
    const int o = s < 0 ? -1 : (s >= B ? 1 : 0);
    s -= o * B;
    return ((unsigned)((o + 1) * DIG) << 20) | (unsigned)(s * STRIDE);
}

// Branch-free pull of every population of cell l of a block whose sources all exist (or read
// the zero block): nboff_s holds the element offsets of the 27 neighbour blocks.
template <class M, int ST, int BX, int BY, int BZ>
__device__ __forceinline__ void gather_fast(const LevelDev& L, int rd, int l, const unsigned* nboff_s,
                                            const ModelDev& m, Cell<M, ST>& c) {
    constexpr int BS = BX * BY * BZ;
    const int lx = l % BX, ly = (l / BX) % BY, lz = l / (BX * BY);
#pragma unroll
    for (int q = 0; q < M::Q; ++q) {
        // one packed term per axis (neighbour digit << 20 | local offset), summed: the terms
        // depend on a single velocity component each and are shared between q
        const unsigned P = axis_term<BX, 1, 1>(lx, M::cx(q)) + axis_term<BY, BX, 3>(ly, M::cy(q)) +
                           axis_term<BZ, BX * BY, 9>(lz, M::cz(q));
        const unsigned i = nboff_s[P >> 20] + (unsigned)(q * BS) + (P & 0xFFFFFu);
        c.f[q] = Store<ST>::template load<M::DEV>(L.f[rd], i, ref_f<M, ST>(m, q));
        if constexpr (M::HAS_G) c.g[q] = Store<ST>::template load<false>(L.g[rd], i, ref_g<M, ST>(m, q));
    }
}

// Coalescence (Eq. coalescence) of every unknown population of every coarse ghost of the
// block, shared out over all the block's threads: the (ghost, population) pairs are numbered by
// a block prefix sum and thread t takes pairs t, t + BS, ...; each pair's 2^D children are
// loaded together and summed in child order.  Result: out[q * BS + cell].
template <class M, int ST, int BX, int BY, int BZ>
__device__ __forceinline__ void coalesce_block(const StepArgs& a, int lev, long long b, int l, unsigned long long umask,
                                               long long child, bool corner, typename Store<ST>::T* out, int* s_cnt,
                                               unsigned long long* s_um, int* s_child, unsigned char* s_corner,
                                               int* s_warp) {
    using T = typename Store<ST>::T;
    constexpr int BS = BX * BY * BZ;
    constexpr int NW = BS / 32;
    constexpr int NK = (M::D == 3) ? 8 : 4;
    s_um[l] = umask;
    s_child[l] = (int)child;
    s_corner[l] = corner ? 1 : 0;
    // block exclusive prefix sum of the pair counts
    const int n = __popcll(umask);
    const int lane = l & 31, w = l >> 5;
    int x = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    int base = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j)
        if (j < w) base += s_warp[j];
    s_cnt[l] = base + x - n;
    if (l == BS - 1) s_cnt[BS] = base + x;
    __syncthreads();
    const int P = s_cnt[BS];
    if (P == 0) return;
    const LevelDev& F = a.lv[lev - 1];
    const int rdf = a.rd[lev - 1];
#pragma unroll 1
    for (int p = l; p < P; p += BS) {
        int lo = 0, hi = BS;                    // owner: the largest o with s_cnt[o] <= p
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_cnt[mid] <= p) lo = mid;
            else hi = mid;
        }
        // the r-th set bit of the owner's mask (0-based), 32 bits at a time
        const unsigned long long m = s_um[lo];
        const int r = p - s_cnt[lo];
        const unsigned m0 = (unsigned)m, m1 = (unsigned)(m >> 32);
        const int c0 = __popc(m0);
        unsigned w = r < c0 ? m0 : m1;
        const int rr = r < c0 ? r : r - c0;          // < popc(w): w keeps a set bit below
        for (int i = 0; i < rr; ++i) w &= w - 1;
        const int q = (r < c0 ? 0 : 32) + __ffs((int)w) - 1;
        const int cx = M::cx(q), cy = M::cy(q), cz = M::cz(q);
        const long long ch0 = s_child[lo];
        const bool cor = s_corner[lo] != 0;
        T own = T(0), vg;
        if (cor) {
            // the ghost's own streamed population, for children whose history left the finer level
            const LevelDev& C = a.lv[lev];
            const long long sc = src_cell_g<BX, BY, BZ>(C.nbr, b * BS + lo, cx, cy, cz);
            load_pop<M, ST, BS>(C, a.rd[lev], sc, q, a.m, own, vg);
        }
        T v[NK];
#pragma unroll
        for (int kk = 0; kk < NK; ++kk) {
            const long long ch = ch0 + (kk & 1) + ((kk >> 1) & 1) * BX + ((kk >> 2) & 1) * BX * BY;
            if (cor && history_leaves<M, BX, BY, BZ>(F, ch, cx, cy, cz)) {
                v[kk] = own;
                continue;
            }
            const long long s = src_cell_g<BX, BY, BZ>(F.nbr, ch, cx, cy, cz);
            load_pop<M, ST, BS>(F, rdf, s, q, a.m, v[kk], vg);
        }
        T sf = 0;
#pragma unroll
        for (int kk = 0; kk < NK; ++kk) sf += v[kk];
        out[q * BS + lo] = sf / T(NK);
    }
}

// Far-field relaxation of Eq. relaxation_pressure, before the collision of a weakly compressible
// cell (populations held as deviations from w rho_ref): rho' = rho (1 - sigma) + sigma rho_inf,
// sigma ramping linearly from 0 at r0 to sigma_max at r1 (distance of the cell centre from the
// centre, finest units).  The equilibrium is linear in rho at fixed u, so f_eq(rho', u) -
// f_eq(rho, u) = (rho' - rho) E(u) with E the equilibrium of unit density: velocity and
// non-equilibrium part are kept.
template <class M, int ST, int BX, int BY, int BZ>
__device__ __forceinline__ void relax_far_field(const ModelDev& m, const LevelDev& L, int lev, long long b, int l,
                                                Cell<M, ST>& c) {
    using T = typename Store<ST>::T;
    static_assert(!M::HAS_G && M::DEV, "weakly compressible deviation models");
    const int lx = l % BX, ly = (l / BX) % BY, lz = l / (BX * BY);
    const double h = double(1 << lev);
    const double x = (double(L.bxyz[3 * b] * BX + lx) + 0.5) * h - m.sp_c[0];
    const double y = (double(L.bxyz[3 * b + 1] * BY + ly) + 0.5) * h - m.sp_c[1];
    const double z = M::D == 3 ? (double(L.bxyz[3 * b + 2] * BZ + lz) + 0.5) * h - m.sp_c[2] : 0.0;
    const double r = sqrt(x * x + y * y + z * z);
    if (!(r > m.sp_r0)) return;
    const double sigma = (r >= m.sp_r1 ? 1.0 : (r - m.sp_r0) / (m.sp_r1 - m.sp_r0)) * m.sp_smax;
    T drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int q = 0; q < M::Q; ++q) {
        drho += c.f[q];
        if (M::cx(q)) jx += T(M::cx(q)) * c.f[q];
        if (M::cy(q)) jy += T(M::cy(q)) * c.f[q];
        if (M::cz(q)) jz += T(M::cz(q)) * c.f[q];
    }
    const T rho = T(m.rho_ref) + drho;
    const T ux = jx / rho, uy = jy / rho, uz = jz / rho;
    const T dr = T(sigma * (m.sp_rho_inf - double(rho)));
    T E[M::Q];
    if constexpr (hermite_weak<M>::value) M::template feq_dev<T>(T(1), ux, uy, T(0), E);
    else weak_feq_dev<M::D, T>(T(1), ux, uy, uz, T(0), E);
#pragma unroll
    for (int q = 0; q < M::Q; ++q) c.f[q] += dr * E[q];
}

// Staging of a block's coarse-ghost post-collision states for the cooperative explosion:
// populations [q][cell], the finer level's block under each octant of the block (-1: none)
// and a coarse-ghost flag per cell.  Empty where the explosion is written per cell.
template <class T, int Q, int BS, bool ON>
struct ExplodeStage {
    T f[Q * BS];
    int fb[8];
    unsigned char cg[BS];
};
template <class T, int Q, int BS>
struct ExplodeStage<T, Q, BS, false> {};
template <class T, int Q, int BS>
__device__ __forceinline__ const T* stage_ptr(const ExplodeStage<T, Q, BS, true>& s) { return s.f; }
template <class T, int Q, int BS>
__device__ __forceinline__ const T* stage_ptr(const ExplodeStage<T, Q, BS, false>&) { return nullptr; }

// One block of cells of the iteration described by a (bid: the block's index in the
// iteration's FAST or general list, over all active levels).
template <class M, int ST, int BX, int BY, int BZ, bool FAST>
__device__ __forceinline__ void step_block(const StepArgs& a, long long bid, int* nbr_s, unsigned long long* s_nstat) {
    using T = typename Store<ST>::T;
    constexpr int BS = BX * BY * BZ;
    // single-distribution models explode through shared memory: each coarse ghost's 2^D
    // children are written by the threads that own those slots of the finer blocks, in whole
    // rows, instead of 2^D scattered stores per population from the ghost's own thread
    constexpr bool COOP = !FAST && !M::HAS_G;
    __shared__ ExplodeStage<T, M::Q, BS, COOP> sx;
    long long i;
    const int lev = find_level_list(a, FAST ? 0 : 1, bid, &i);
    const LevelDev& L = a.lv[lev];
    const int entry = L.blist[FAST ? 0 : 1][i];
    // FAST list entries carry a streaming-block bit: such blocks hold fine ghosts, absent slots
    // and Neumann boundary cells (partner in the block) besides record-free fluid cells, so the
    // cell types are read and a missing neighbour block reads the zero-population block nb
    const long long b = FAST ? (long long)(entry >> 2) : (long long)entry;
    const bool streaming = FAST && (entry & 1);
    const int l = threadIdx.x;
    // element offset of each neighbour block's populations (the zero block for a missing one)
    __shared__ unsigned nboff_s[27];
    if (l < 27) {
        const int v = L.nbr[b * 27 + l];
        nbr_s[l] = (FAST && v < 0) ? (int)L.nb : v;
        nboff_s[l] = (unsigned)(v < 0 ? L.nb : v) * (unsigned)(M::Q * BS);
    }
    if (M::HAS_LAM && l < 19) s_nstat[l] = 0ull;
    if constexpr (COOP) {
        if (l < 8) sx.fb[l] = -1;
        sx.cg[l] = 0;
    }
    __syncthreads();
    const long long cell = b * BS + l;
    const int rd = a.rd[lev], wr = rd ^ 1;
    const int type = (FAST && !streaming) ? (int)C_FLUID : (int)L.type[cell];
    const bool work = !(type == C_ABSENT || type == C_SOLID || (type == C_FGHOST && a.sync_fg[lev]));
    if constexpr (COOP) {
        __shared__ int s_cnt[BS + 1], s_child[BS], s_warp[BS / 32];
        __shared__ unsigned long long s_um[BS];
        __shared__ unsigned char s_corner[BS];
        unsigned long long um = 0ull;
        long long child = 0;
        bool corner = false;
        if (type == C_CGHOST) {
            const CellRecDev rec = L.recs[L.rec_id[cell]];
            um = rec.mask;
            child = rec.a;
            corner = (rec.b & 1) != 0;
        }
        coalesce_block<M, ST, BX, BY, BZ>(a, lev, b, l, um, child, corner, sx.f, s_cnt, s_um, s_child, s_corner,
                                          s_warp);
        __syncthreads();
    }
    int iters = -1;
    if (work) {
        Cell<M, ST> c;
        int conv = 1, conv2 = 1;
        // fluid cells without a record (no bounce-back link) have every source live: gather
        // them branch-free also inside the general blocks
        if (FAST || (type == C_FLUID && L.rec_id[cell] < 0)) {
            // a Neumann boundary cell of an interior block pulls at its partner, which lies in
            // the block (Appendix A.3: the partner's streamed state, multipliers included)
            long long src = cell;
            int ls = l;
            if (FAST && (entry & 2) && type == C_BC) {
                src = L.recs[L.rec_id[cell]].a;
                ls = int(src - b * BS);
                __builtin_assume(ls >= 0 && ls < BS);
            }
            gather_fast<M, ST, BX, BY, BZ>(L, rd, ls, nboff_s, a.m, c);
            if constexpr (M::HAS_LAM) {
#pragma unroll
                for (int j = 0; j < 8; ++j) c.lam[j] = L.lam[((long long)rd * 8 + j) * L.ncell + src];
            }
        } else if constexpr (!FAST) {
            assemble<M, ST, BX, BY, BZ, MODE_STEP>(a, lev, b, l, type, false, nbr_s, c, &conv, stage_ptr(sx));
        }
        // interior kernel, binary16 deviations, recursive regularization: the collision writes
        // the storage value directly (fine ghosts, which do not collide, are scaled instead)
        constexpr bool REL = FAST && ST == ST_F16DEV && !M::HAS_G && M::RR && M::DEV;
        if constexpr (!M::HAS_G && M::DEV && !FAST) {   // every block takes this kernel then
            if (a.m.sponge_on && type != C_FGHOST) relax_far_field<M, ST, BX, BY, BZ>(a.m, L, lev, b, l, c);
        }
        if (type != C_FGHOST) {
            const int it = collide<M, ST, REL>(a.m, L, c, &conv2);
            if (M::HAS_LAM) iters = it + (conv2 ? 0 : 1000);
            if (!conv || !conv2) set_status(a.status, -6);
        } else if constexpr (REL) {
#pragma unroll
            for (int q = 0; q < M::Q; ++q) c.f[q] *= inv_ref_f<M, ST>(a.m, q);
        }
        // fine ghosts stream purely: stored as gathered (post-collision = pre-collision)
        if constexpr (REL) {
#pragma unroll
            for (int q = 0; q < M::Q; ++q)
                ((__half*)L.f[wr])[pidx<BX * BY * BZ, M::Q>(cell, q)] = __float2half_rn(c.f[q]);
        } else {
#pragma unroll
            for (int q = 0; q < M::Q; ++q) store_pop<M, ST, BX * BY * BZ>(L, wr, cell, q, a.m, c.f[q], M::HAS_G ? c.g[q] : T(0));
        }
        if constexpr (M::HAS_LAM) {
#pragma unroll
            for (int j = 0; j < 8; ++j) L.lam[((long long)wr * 8 + j) * L.ncell + cell] = c.lam[j];
        }
        if constexpr (COOP) {
            if (type == C_CGHOST) {
                const int lx = l % BX, ly = (l / BX) % BY, lz = l / (BX * BY);
#pragma unroll
                for (int q = 0; q < M::Q; ++q) sx.f[q * BS + l] = c.f[q];
                sx.cg[l] = 1;
                const long long child = L.recs[L.rec_id[cell]].a;
                sx.fb[(2 * lx) / BX + 2 * ((2 * ly) / BY) + 4 * ((2 * lz) / BZ)] = (int)(child / BS);
            }
        } else if constexpr (!FAST) {
            if (type == C_CGHOST) {
                // uniform explosion (Eq. explosion_uniform) into every child's slot of the buffer
                // the finer level writes at this iteration
                const LevelDev& F = a.lv[lev - 1];
                const int wrf = a.rd[lev - 1] ^ 1;
                const long long child = L.recs[L.rec_id[cell]].a;
                constexpr int NK = (M::D == 3) ? 8 : 4;
#pragma unroll 1
                for (int kk = 0; kk < NK; ++kk) {
                    const long long ch = child + (kk & 1) + ((kk >> 1) & 1) * BX + ((kk >> 2) & 1) * BX * BY;
#pragma unroll
                    for (int q = 0; q < M::Q; ++q) store_pop<M, ST, BX * BY * BZ>(F, wrf, ch, q, a.m, c.f[q], M::HAS_G ? c.g[q] : T(0));
                    if constexpr (M::HAS_LAM) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) F.lam[((long long)wrf * 8 + j) * F.ncell + ch] = c.lam[j];
                    }
                }
            }
        }
    }
    if constexpr (COOP) {
        // uniform explosion (Eq. explosion_uniform): every child of every coarse ghost of this
        // block receives the ghost's post-collision populations in the buffer the finer level
        // writes at this iteration
        if (__syncthreads_or(work && type == C_CGHOST)) {
            const LevelDev& F = a.lv[lev - 1];
            const int wrf = a.rd[lev - 1] ^ 1;
            const int fx = l % BX, fy = (l / BX) % BY, fz = l / (BX * BY);
            constexpr int NOCT = (M::D == 3) ? 8 : 4;
#pragma unroll 1
            for (int oct = 0; oct < NOCT; ++oct) {
                const int fb = sx.fb[oct];
                if (fb < 0) continue;
                const int px = ((oct & 1) * BX + fx) >> 1;
                const int py = (((oct >> 1) & 1) * BY + fy) >> 1;
                const int pz = (((oct >> 2) & 1) * BZ + fz) >> 1;
                const int p = (pz * BY + py) * BX + px;
                if (!sx.cg[p]) continue;
                const long long ch = (long long)fb * BS + l;
#pragma unroll
                for (int q = 0; q < M::Q; ++q) store_pop<M, ST, BS>(F, wrf, ch, q, a.m, sx.f[q * BS + p], T(0));
            }
        }
    }
    if constexpr (M::HAS_LAM) {
        if (iters >= 0) {
            const int nc = iters >= 1000;
            const int it = iters - 1000 * nc;
            atomicAdd(&s_nstat[0], (unsigned long long)it);
            atomicAdd(&s_nstat[1], 1ull);
            if (nc) atomicAdd(&s_nstat[2], 1ull);
            atomicAdd(&s_nstat[3 + (it < 15 ? it : 15)], 1ull);
        }
        __syncthreads();
        if (l < 19 && s_nstat[l]) atomicAdd(&a.nstat[l], s_nstat[l]);
    }
}

// occupancy target (resident 128-thread blocks per SM); MINB > 0 overrides the model's
template <class M, int ST, bool FAST, int MINB>
constexpr int step_min_blocks(int threads) {
    return (MINB > 0 ? MINB : ((FAST ? M::MINB_FAST : M::MINB_GEN) / (ST == ST_F64 ? 2 : 1))) * 128 / threads;
}

template <class M, int ST, int BX, int BY, int BZ, bool FAST, int MINB>
__global__ void __launch_bounds__(BX * BY * BZ, step_min_blocks<M, ST, FAST, MINB>(BX * BY * BZ))
k_step(const StepArgs a) {
    __shared__ int nbr_s[27];
    __shared__ unsigned long long s_nstat[19];
    step_block<M, ST, BX, BY, BZ, FAST>(a, blockIdx.x, nbr_s, s_nstat);
}

// Batched form: the blocks of several independent cases of one iteration in one launch.
// args[k] describes case k at this iteration; off[k] .. off[k + 1] are its blocks in the
// launch (off[n] = grid size).  A block finds its case by binary search.
template <class M, int ST, int BX, int BY, int BZ, bool FAST, int MINB>
__global__ void __launch_bounds__(BX * BY * BZ, step_min_blocks<M, ST, FAST, MINB>(BX * BY * BZ))
k_step_batch(const StepArgs* __restrict__ args, const long long* __restrict__ off, int n) {
    __shared__ int nbr_s[27];
    __shared__ unsigned long long s_nstat[19];
    const long long bid = blockIdx.x;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bid >= off[mid]) lo = mid;
        else hi = mid;
    }
    step_block<M, ST, BX, BY, BZ, FAST>(args[lo], bid - off[lo], nbr_s, s_nstat);
}

// ------------------------------------------------------------------ staged binary16 interior kernel
// Interior (simple and streaming) blocks of the D3Q27 regularized model in binary16 deviation
// storage, with the pull staged in shared memory and two cells per thread.  A block's cells are
// BY * BZ = 16 rows of 8 cells, and one row of one population is 16 bytes of storage, so the pull
// of population q for the whole block is 16 row copies (cp.async, 16 bytes each): destination
// row (ly, lz) receives the row (ly - xi_y, lz - xi_z) of whichever block holds it (its "own-side"
// row).  When xi_x != 0 one cell of each row sources from the x-neighbour block: a 4-byte copy of
// that neighbour's edge pair (elements 6, 7 of the x-1 neighbour for xi_x = +1, elements 0, 1 of
// the x+1 neighbour for xi_x = -1) lands in a word per row after the 16 own-side rows.  Each
// population's staged region is at a fixed offset, and each thread reads it at offsets fixed per
// thread, so the gather is one shared-memory load per population and cell.  A thread owns the
// x-neighbours (2k, 2k + 1) of a row: the collision (rr_rel_q27) runs on both at once in packed
// FP32 pairs, directly on the stored relative deviations, and each population of the pair is
// stored as one 32-bit word.  A thread block takes NB cell blocks (a stride of the grid apart) in
// turn, with two staging buffers: the rows of the next cell block and the neighbour list of the one
// after are copied while the current one collides, so the copies' latency is hidden behind
// arithmetic.  A Neumann boundary cell pulls its partner's populations, so it receives the
// partner's stored result after a block barrier (only in blocks whose list entry has bit 1).
template <class M, int ST, int BX, int BY, int BZ>
struct staged_f16 : std::bool_constant<ST == ST_F16DEV && M::D == 3 && M::Q == 27 && !M::HAS_G && !M::HAS_LAM &&
                                       M::DEV && M::RR && !hermite_weak<M>::value && weak_var<M>::value == 0 &&
                                       BX == 8 && BY * BZ == 16> {};

__device__ __forceinline__ void cp_async16(unsigned smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(unsigned smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// staged bytes of population q (16 own-side rows of 16 bytes, and 16 edge words when xi_x != 0)
// and its offset in a staging buffer
template <class M>
__host__ __device__ constexpr int stg_bytes(int q) { return M::cx(q) == 0 ? 256 : 320; }
template <class M>
__host__ __device__ constexpr int stg_off(int q) {
    int o = 0;
    for (int k = 0; k < q; ++k) o += stg_bytes<M>(k);
    return o;
}

// Copy of population Q for destination row r (y, z terms ty, tz of that row) and part p
// (0: the own-side row, 1: the x-neighbour's edge word, only for xi_x != 0); nbo: the 27
// neighbour blocks' element offsets.
template <class M, int BX, int BY, int BZ, int Q>
__device__ __forceinline__ void stage_pop(const char* fsrc, const unsigned* nbo, unsigned sbase, int r, int p,
                                          const unsigned* ty, const unsigned* tz) {
    constexpr int BS = BX * BY * BZ;
    constexpr int cx = M::cx(Q), cy = M::cy(Q), cz = M::cz(Q);
    if (cx == 0 && p) return;
    // neighbour digit of x: 1 (own column of blocks) or 1 - xi_x (the x-neighbour, at -xi_x)
    const unsigned P = ((unsigned)(p ? 1 - cx : 1) << 20) + ty[cy + 1] + tz[cz + 1];
    const unsigned idx = nbo[P >> 20] + (unsigned)(Q * BS) + (P & 0xFFFFFu);
    if (p == 0) {
        cp_async16(sbase + (unsigned)(stg_off<M>(Q) + r * 16), fsrc + 2ull * idx);
    } else {
        // elements 6, 7 of the x-1 neighbour's row (xi_x = +1) or 0, 1 of the x+1 neighbour's
        cp_async4(sbase + (unsigned)(stg_off<M>(Q) + 256 + r * 4), fsrc + 2ull * (idx + (cx == 1 ? BX - 2 : 0)));
    }
}
template <class M, int BX, int BY, int BZ, int NW, int W, int... I>
__device__ __forceinline__ void stage_warp(std::integer_sequence<int, I...>, const char* fsrc, const unsigned* nbo,
                                           unsigned sbase, int r, int p, const unsigned* ty, const unsigned* tz) {
    (
        [&] {
            if constexpr (W + NW * I < M::Q) stage_pop<M, BX, BY, BZ, W + NW * I>(fsrc, nbo, sbase, r, p, ty, tz);
        }(),
        ...);
}

// The staged kernel's variants, by the occupancy code of the direct kernel they stand in for:
// ten resident thread blocks per SM (96 registers, 16.6 KB of shared memory each) taking 4 (model
// default), 8 (targets of 8 direct blocks) or 16 (6) cell blocks each.
constexpr int staged_min_blocks(int) { return 10; }
constexpr int staged_nb(int minb) { return minb == 8 ? 8 : (minb == 6 ? 16 : 4); }

template <class M, int ST, int BX, int BY, int BZ, int MINB, int NB>
__global__ void __launch_bounds__(BX * BY * BZ / 2, staged_min_blocks(MINB))
k_step_staged(const StepArgs a) {
    constexpr int BS = BX * BY * BZ;
    constexpr int NT = BS / 2;                              // threads: two cells each
    constexpr int NW = NT / 32;                             // warps
    constexpr int ROWS = BY * BZ;
    static_assert(NW == 2 && ROWS == 16, "two warps; a warp's 32 lanes cover 16 rows x 2 parts");
    static_assert(NB >= 1 && NB <= NT, "cell blocks per thread block");
    constexpr int SB = stg_off<M>(M::Q);                    // bytes of one staging buffer
    __shared__ __align__(16) unsigned char stg[2][SB];
    __shared__ int nbr3[3][28];                             // neighbour lists of three cell blocks
    __shared__ unsigned nbo[27];                            // element offsets, cell block being staged
    __shared__ int ent_s[NB], lev_s[NB];
    const long long n = a.list_off[0][a.n_active];
    const int t = threadIdx.x;
    const int lane = t & 31, w = t >> 5;
    const int r = lane & (ROWS - 1), p = lane >> 4;
    // slot j: cell block blockIdx.x + j * gridDim.x of this iteration's interior list
    auto slot_ok = [&](int j) { return (long long)blockIdx.x + (long long)j * gridDim.x < n; };
    if (t < NB) {
        const long long g = (long long)blockIdx.x + (long long)t * gridDim.x;
        int lev = 0, e = 0;
        if (g < n) {
            long long i;
            lev = find_level_list(a, 0, g, &i);
            e = a.lv[lev].blist[0][i];
        }
        ent_s[t] = e;
        lev_s[t] = lev;
    }
    __syncthreads();
    auto nbr_src = [&](int j) { return a.lv[lev_s[j]].nbr + (long long)(ent_s[j] >> 2) * 27 + t; };
    if (t < 27) nbr3[0][t] = *nbr_src(0);
    if (NB > 1 && t < 27 && slot_ok(1)) cp_async4((unsigned)__cvta_generic_to_shared(&nbr3[1][t]), nbr_src(1));
    unsigned ty[3], tz[3];
    {
        const int ry = r % BY, rz = r / BY;
#pragma unroll
        for (int c = -1; c <= 1; ++c) {
            ty[c + 1] = axis_term<BY, BX, 3>(ry, c);
            tz[c + 1] = axis_term<BZ, BX * BY, 9>(rz, c);
        }
    }
    // copies of the rows of slot j into buffer j & 1 (its neighbour list landed in nbr3[j % 3])
    auto stage = [&](int j) {
        const LevelDev& L = a.lv[lev_s[j]];
        if (t < 27) {
            const int v = nbr3[j % 3][t];
            nbo[t] = (unsigned)(v < 0 ? L.nb : v) * (unsigned)(M::Q * BS);
        }
        __syncthreads();
        const char* fsrc = (const char*)L.f[a.rd[lev_s[j]]];
        const unsigned sbase = (unsigned)__cvta_generic_to_shared(stg[j & 1]);
        using Seq = std::make_integer_sequence<int, (27 + NW - 1) / NW>;
        if (w == 0) stage_warp<M, BX, BY, BZ, NW, 0>(Seq{}, fsrc, nbo, sbase, r, p, ty, tz);
        else stage_warp<M, BX, BY, BZ, NW, 1>(Seq{}, fsrc, nbo, sbase, r, p, ty, tz);
    };
    __syncthreads();
    stage(0);
    cp_async_commit();
    // cells (2k, row) and (2k + 1, row) of each cell block
    const int k2 = 2 * (t % (BX / 2)), row = t / (BX / 2);
    const int l0 = k2 + BX * row;
#pragma unroll 1
    for (int j = 0; j < NB && slot_ok(j); ++j) {
        cp_async_wait_all();
        __syncthreads();          // slot j's rows and slot j + 1's neighbour list are in place
        if (j + 2 < NB && t < 27 && slot_ok(j + 2))
            cp_async4((unsigned)__cvta_generic_to_shared(&nbr3[(j + 2) % 3][t]), nbr_src(j + 2));
        if (j + 1 < NB && slot_ok(j + 1)) stage(j + 1);
        cp_async_commit();
        // collide slot j from buffer j & 1
        const int lev = lev_s[j];
        const LevelDev& L = a.lv[lev];
        const long long b = (long long)(ent_s[j] >> 2);
        const bool streaming = ent_s[j] & 1;
        const long long cell = b * BS + l0;
        bool work0 = true, work1 = true, fg0 = false, fg1 = false, bc0 = false, bc1 = false;
        if (streaming) {
            const int t0 = L.type[cell], t1 = L.type[cell + 1];
            work0 = !(t0 == C_ABSENT || t0 == C_SOLID || (t0 == C_FGHOST && a.sync_fg[lev]));
            work1 = !(t1 == C_ABSENT || t1 == C_SOLID || (t1 == C_FGHOST && a.sync_fg[lev]));
            fg0 = t0 == C_FGHOST;
            fg1 = t1 == C_FGHOST;
            bc0 = t0 == C_BC;
            bc1 = t1 == C_BC;
        }
        // byte offsets of the pair's sources within a population's staged region: xi_x = 0 (both),
        // xi_x = +1 (x = 2k - 1: the edge word's upper half for k = 0; x = 2k), xi_x = -1 (x = 2k + 1;
        // x = 2k + 2: the edge word's lower half for the last pair)
        const unsigned char* buf = stg[j & 1];
        const int o0 = row * 16 + 2 * k2;
        const int op0 = k2 == 0 ? 256 + row * 4 + 2 : o0 - 2, op1 = o0;
        const int om0 = o0 + 2, om1 = k2 == BX - 2 ? 256 + row * 4 : o0 + 4;
        __half* out = (__half*)L.f[a.rd[lev] ^ 1];
        const long long base = b * (long long)(M::Q * BS) + l0;
        // fine ghosts stream purely: their staged values are stored as gathered
        if (streaming && ((work0 && fg0) || (work1 && fg1))) {
#pragma unroll
            for (int q = 0; q < M::Q; ++q) {
                const unsigned char* sq = buf + stg_off<M>(q);
                const int a0 = M::cx(q) == 0 ? o0 : (M::cx(q) == 1 ? op0 : om0);
                const int a1 = M::cx(q) == 0 ? o0 + 2 : (M::cx(q) == 1 ? op1 : om1);
                if (work0 && fg0) out[base + q * BS] = *(const __half*)(sq + a0);
                if (work1 && fg1) out[base + q * BS + 1] = *(const __half*)(sq + a1);
            }
        }
        const bool c0 = work0 && !fg0 && !bc0, c1 = work1 && !fg1 && !bc1;
        if (c0 || c1) {
            F2 h[M::Q];
#pragma unroll
            for (int q = 0; q < M::Q; ++q) {
                const unsigned char* sq = buf + stg_off<M>(q);
                if (M::cx(q) == 0) {
                    h[q].v = __half22float2(*(const __half2*)(sq + o0));    // 4-byte aligned pair
                } else {
                    const int a0 = M::cx(q) == 1 ? op0 : om0, a1 = M::cx(q) == 1 ? op1 : om1;
                    h[q].v = make_float2(__half2float(*(const __half*)(sq + a0)), __half2float(*(const __half*)(sq + a1)));
                }
            }
            const bool both = c0 && c1;
            rr_rel_q27<F2>(h, 1.0f - L.omega_f, [&](int q, F2 v) {
                if (both) {
                    *(__half2*)(out + base + q * BS) = __float22half2_rn(v.v);
                } else {
                    if (c0) out[base + q * BS] = __float2half_rn(v.v.x);
                    if (c1) out[base + q * BS + 1] = __float2half_rn(v.v.y);
                }
            });
        }
        // Neumann boundary cells (Appendix A.3) pull the partner's populations, in the block,
        // so their collided state is the partner's: copied once every partner has been stored
        if (ent_s[j] & 2) {
            __syncthreads();
#pragma unroll 1
            for (int i = 0; i < 2; ++i) {
                if (!(i ? bc1 : bc0)) continue;
                const long long P = L.recs[L.rec_id[cell + i]].a;
                const long long pb = b * (long long)(M::Q * BS) + (P - b * BS);
#pragma unroll
                for (int q = 0; q < M::Q; ++q) out[base + q * BS + i] = out[pb + q * BS];
            }
        }
    }
    cp_async_wait_all();
}

// ------------------------------------------------------------------ AA-pattern streaming
// In-place streaming with one population buffer, on single-level grids.  Two layouts alternate:
//   L1 (after an even number of iterations): slot (x, qbar) holds the pre-collision f_q(x);
//   L0 (after an odd number): slot (x, q) holds the post-collision f*_q(x), the layout the
//       two-buffer path gathers from, so readouts and ledgers read it unchanged.
// Even iteration (L1 -> L0): a cell reads its own slots reversed and writes its own slots.
// Odd iteration (L0 -> L1): cell x gathers f_q(x) = slot (x - xi_q, q) and writes f*_p(x) to
// slot (x + xi_p, pbar), the slot it read for q = pbar: every slot is read and then written by
// one thread, so no two threads touch a slot.  A blocked link q (solid or wall) reads and writes
// the cell's own slot qbar, with Ladd's term at moving walls; the bounced value then already sits
// where the even iteration reads it.

// Boundary-layer cell of an equilibrium Dirichlet face (imposed rho, u, T): its pre-collision
// state is the equilibrium (the face kinds that read an interior partner are not offered with
// AA streaming).
template <class M, int ST>
__device__ __forceinline__ void bc_equilibrium(const StepArgs& a, const LevelDev& L, long long cell,
                                               Cell<M, ST>& c, int* conv) {
    using T = typename Store<ST>::T;
    const CellRecDev rec = L.recs[L.rec_id[cell]];
    const FaceDev& fd = a.m.faces[rec.b >> 4];
    *conv = 1;
    if constexpr (!M::HAS_G) {
        if constexpr (hermite_weak<M>::value) M::template feq_dev<T>(T(fd.rho), T(fd.u[0]), T(fd.u[1]), T(a.m.rho_ref), c.f);
        else weak_feq_dev<M::D, T>(T(fd.rho), T(fd.u[0]), T(fd.u[1]), T(fd.u[2]), T(a.m.rho_ref), c.f);
    } else {
        int it = 0;
        M::template feq<ST>(a.m, T(fd.rho), T(fd.u[0]), T(fd.u[1]), T(fd.T), c.lam, c.f, &it, conv);
        const T gfac = T((2.0 * a.m.Cv - M::D) * fd.T);
#pragma unroll
        for (int q = 0; q < M::Q; ++q) c.g[q] = gfac * c.f[q];
    }
}

template <class M, int ST, int BX, int BY, int BZ, bool ODD>
__global__ void __launch_bounds__(BX * BY * BZ, step_min_blocks<M, ST, true, 0>(BX * BY * BZ))
k_step_aa(const StepArgs a) {
    using T = typename Store<ST>::T;
    constexpr int BS = BX * BY * BZ;
    __shared__ int nbr_s[27];
    __shared__ unsigned nboff_s[27];
    __shared__ unsigned long long s_nstat[19];
    const LevelDev& L = a.lv[0];
    const long long b = blockIdx.x;
    const int l = threadIdx.x;
    if (l < 27) {
        const int v = L.nbr[b * 27 + l];
        nbr_s[l] = v;
        nboff_s[l] = (unsigned)(v < 0 ? L.nb : v) * (unsigned)(M::Q * BS);
    }
    if (M::HAS_LAM && l < 19) s_nstat[l] = 0ull;
    __syncthreads();
    const long long cell = b * BS + l;
    const bool simple = L.bflag[b] == 1;
    const int type = simple ? (int)C_FLUID : (int)L.type[cell];
    int iters = -1;
    if (type == C_FLUID || type == C_BC) {
        const int lx = l % BX, ly = (l / BX) % BY, lz = l / (BX * BY);
        unsigned long long bmask = 0ull;
        bool walls = false;
        if (!simple && type == C_FLUID) {
            const int r = L.rec_id[cell];
            if (r >= 0) {
                const CellRecDev rec = L.recs[r];
                bmask = rec.mask;
                walls = (rec.b & 2) != 0;
            }
        }
        Cell<M, ST> c;
        int conv = 1, conv2 = 1;
        if constexpr (M::HAS_LAM) {
#pragma unroll
            for (int j = 0; j < 8; ++j) c.lam[j] = L.lam[(long long)j * L.ncell + cell];
        }
        if (type == C_BC) {
            bc_equilibrium<M, ST>(a, L, cell, c, &conv);
        } else if (ODD && simple) {
            gather_fast<M, ST, BX, BY, BZ>(L, 0, l, nboff_s, a.m, c);     // every source exists
        } else {
#pragma unroll
            for (int q = 0; q < M::Q; ++q) {
                T gv = T(0);
                if (!ODD || (bmask >> q & 1ull)) {
                    load_pop<M, ST, BS>(L, 0, cell, M::Q - 1 - q, a.m, c.f[q], gv);
                    if constexpr (ODD && !M::HAS_G) {
                        if (walls) c.f[q] += T(wall_term<M, BX, BY, BZ>(a.m, L, b, l, q));
                    }
                } else {
                    const long long s = src_cell<BX, BY, BZ>(nbr_s, b, lx, ly, lz, M::cx(q), M::cy(q), M::cz(q));
                    load_pop<M, ST, BS>(L, 0, s, q, a.m, c.f[q], gv);
                }
                if constexpr (M::HAS_G) c.g[q] = gv;
            }
        }
        if constexpr (!M::HAS_G && M::DEV) {
            if (a.m.sponge_on) relax_far_field<M, ST, BX, BY, BZ>(a.m, L, 0, b, l, c);
        }
        const int it = collide<M, ST, false>(a.m, L, c, &conv2);
        if (M::HAS_LAM) iters = it + (conv2 ? 0 : 1000);
        if (!conv || !conv2) set_status(a.status, -6);
#pragma unroll
        for (int p = 0; p < M::Q; ++p) {
            const T gp = M::HAS_G ? c.g[p] : T(0);
            if (!ODD) {
                store_pop<M, ST, BS>(L, 0, cell, p, a.m, c.f[p], gp);
            } else if (simple) {
                // slot (x + xi_p, pbar): the source of link pbar, by the packed per-axis offsets
                const int pb = M::Q - 1 - p;
                const unsigned P = axis_term<BX, 1, 1>(lx, M::cx(pb)) + axis_term<BY, BX, 3>(ly, M::cy(pb)) +
                                   axis_term<BZ, BX * BY, 9>(lz, M::cz(pb));
                const unsigned i = nboff_s[P >> 20] + (unsigned)(pb * BS) + (P & 0xFFFFFu);
                Store<ST>::template store<M::DEV>(L.f[0], i, c.f[p], inv_ref_f<M, ST>(a.m, pb));
                if constexpr (M::HAS_G) Store<ST>::template store<false>(L.g[0], i, gp, inv_ref_g<M, ST>(a.m, pb));
            } else {
                const int pb = M::Q - 1 - p;
                if (bmask >> pb & 1ull) {
                    T v = c.f[p];
                    if constexpr (!M::HAS_G) {
                        if (walls) v += T(wall_term<M, BX, BY, BZ>(a.m, L, b, l, pb));
                    }
                    store_pop<M, ST, BS>(L, 0, cell, p, a.m, v, gp);
                } else {
                    const long long d = src_cell<BX, BY, BZ>(nbr_s, b, lx, ly, lz, M::cx(pb), M::cy(pb), M::cz(pb));
                    if (d >= 0) store_pop<M, ST, BS>(L, 0, d, pb, a.m, c.f[p], gp);
                }
            }
        }
        if constexpr (M::HAS_LAM) {
#pragma unroll
            for (int j = 0; j < 8; ++j) L.lam[(long long)j * L.ncell + cell] = c.lam[j];
        }
    }
    if constexpr (M::HAS_LAM) {
        if (iters >= 0) {
            const int nc = iters >= 1000;
            const int it = iters - 1000 * nc;
            atomicAdd(&s_nstat[0], (unsigned long long)it);
            atomicAdd(&s_nstat[1], 1ull);
            if (nc) atomicAdd(&s_nstat[2], 1ull);
            atomicAdd(&s_nstat[3 + (it < 15 ? it : 15)], 1ull);
        }
        __syncthreads();
        if (l < 19 && s_nstat[l]) atomicAdd(&a.nstat[l], s_nstat[l]);
    }
}

// ------------------------------------------------------------------ readout
// out (FP64, SoA over the level's slots): which = 0 moments (rho, ux, uy, uz, T),
// 1 populations f, 2 populations g, 3 lambda
template <class M, int ST, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ) k_read(const StepArgs a, int lev, int which, double* out) {
    using T = typename Store<ST>::T;
    constexpr int BS = BX * BY * BZ;
    __shared__ int nbr_s[27];
    const LevelDev& L = a.lv[lev];
    const long long b = blockIdx.x;
    const int l = threadIdx.x;
    if (l < 27) nbr_s[l] = L.nbr[b * 27 + l];
    __syncthreads();
    const long long cell = b * BS + l;
    const bool simple = L.bflag[b] == 1;
    const int type = simple ? (int)C_FLUID : (int)L.type[cell];
    if (type == C_ABSENT || type == C_SOLID) return;
    Cell<M, ST> c;
    int conv;
    // which 4..6: the conserved (ledger) state, coarse ghosts with their unknowns coalesced
    if (which >= 4 && which <= 6) assemble<M, ST, BX, BY, BZ, MODE_LEDGER>(a, lev, b, l, type, simple, nbr_s, c, &conv);
    else assemble<M, ST, BX, BY, BZ, MODE_READ>(a, lev, b, l, type, simple, nbr_s, c, &conv);
    // the conserved state is handed on as stored (deviations for the deviation formats), so
    // that a copy is exact
    const bool raw = which >= 4 && which <= 6;
    if (raw) which -= 3;
    if (which == 7) {
        // kinetic sensor eps = (1/V) sum |f - f_eq| / f_eq of the pre-collision state (Eq.
        // DeltaAvg; the refinement criterion of Sec. 8), terms with f_eq <= tiny skipped
        using T = typename Store<ST>::T;
        T rho, u[3], Tt;
        moments<M, ST>(a.m, c, rho, u, Tt);
        T fe[M::Q];
        if constexpr (!M::HAS_G) {
            if constexpr (hermite_weak<M>::value) M::template feq_dev<T>(rho, u[0], u[1], T(a.m.rho_ref), fe);
            else weak_feq_dev<M::D, T>(rho, u[0], u[1], u[2], T(a.m.rho_ref), fe);
        } else {
            int it = 0, cv = 1;
            M::template feq<ST>(a.m, rho, u[0], u[1], Tt, c.lam, fe, &it, &cv);
        }
        double eps = 0.0;
#pragma unroll
        for (int q = 0; q < M::Q; ++q) {
            const double ref = M::DEV ? M::w(q) * a.m.rho_ref : 0.0;
            const double fq = double(c.f[q]) + ref, eq = double(fe[q]) + ref;
            if (eq > 1e-300) eps += fabs(fq - eq) / eq;
        }
        out[cell] = eps / M::Q;
        return;
    }
    if (which == 0) {
        T rho, u[3], Tt;
        moments<M, ST>(a.m, c, rho, u, Tt);
        out[0 * L.ncell + cell] = rho;
        out[1 * L.ncell + cell] = u[0];
        out[2 * L.ncell + cell] = u[1];
        out[3 * L.ncell + cell] = u[2];
        out[4 * L.ncell + cell] = Tt;
    } else if (which == 1) {
#pragma unroll
        for (int q = 0; q < M::Q; ++q)
            out[(long long)q * L.ncell + cell] = (M::DEV && !raw) ? (double)c.f[q] + M::w(q) * a.m.rho_ref : (double)c.f[q];
    } else if (which == 2) {
        if constexpr (M::HAS_G) {
#pragma unroll
            for (int q = 0; q < M::Q; ++q) out[(long long)q * L.ncell + cell] = c.g[q];
        }
    } else if (which == 3) {
        if constexpr (M::HAS_LAM) {
#pragma unroll
            for (int i = 0; i < 8; ++i) out[(long long)i * L.ncell + cell] = c.lam[i];
        }
    }
}

// ------------------------------------------------------------------ ledger (FP64, deterministic)
// Per block: the volume-weighted sums of the cells of the block, reduced in a fixed tree order
// into partial[block * 5 + j]; a second kernel reduces the partials in a fixed order.
template <class M, int ST, int BX, int BY, int BZ>
__device__ __forceinline__ void ledger_block(const StepArgs& a, long long bid, double* partial) {
    constexpr int BS = BX * BY * BZ;
    __shared__ int nbr_s[27];
    __shared__ unsigned nboff_s[27];
    __shared__ double red[5][BS / 32];
    long long b;
    const int lev = find_level(a, bid, &b);
    const LevelDev& L = a.lv[lev];
    const int l = threadIdx.x;
    if (l < 27) {
        const int v = L.nbr[b * 27 + l];
        nbr_s[l] = v;
        nboff_s[l] = (unsigned)(v < 0 ? L.nb : v) * (unsigned)(M::Q * BS);
    }
    __syncthreads();
    const long long cell = b * BS + l;
    const int bf = L.bflag[b];
    const bool simple = bf == 1;
    const int type = simple ? (int)C_FLUID : (int)L.type[cell];
    double v[5] = {0, 0, 0, 0, 0};
    if (type == C_FLUID || type == C_BC || type == C_CGHOST) {
        Cell<M, ST> c;
        int conv;
        // fluid cells of simple and streaming blocks have every source: the branch-free pull
        if (bf != 0 && type == C_FLUID && !a.aa_l1) gather_fast<M, ST, BX, BY, BZ>(L, a.rd[lev], l, nboff_s, a.m, c);
        else assemble<M, ST, BX, BY, BZ, MODE_LEDGER>(a, lev, b, l, type, simple, nbr_s, c, &conv);
        const double V = double(1ll << (lev * M::D));
        // per-cell sums in the arithmetic type of the stored values (the deviations f - w rho_ref
        // of the weak models are small, so FP32 sums keep their absolute error far below the
        // FP64 totals' rounding); the reference part rho_ref (sum w, sum w |xi|^2 / 2) is added in
        // FP64, then the level's cell volume
        using T = typename Store<ST>::T;
        T s[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int q = 0; q < M::Q; ++q) {
            const T fq = c.f[q];
            s[0] += fq;
            if (M::cx(q)) s[1] += T(M::cx(q)) * fq;
            if (M::cy(q)) s[2] += T(M::cy(q)) * fq;
            if (M::cz(q)) s[3] += T(M::cz(q)) * fq;
            const int x2 = M::cx(q) * M::cx(q) + M::cy(q) * M::cy(q) + M::cz(q) * M::cz(q);
            if (x2) s[4] += T(0.5 * x2) * fq;
            if constexpr (M::HAS_G) s[4] += T(0.5) * c.g[q];
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = (double)s[j];
        if constexpr (M::DEV) {
            double e_ref = 0.0;
#pragma unroll
            for (int q = 0; q < M::Q; ++q)
                e_ref += 0.5 * M::w(q) * double(M::cx(q) * M::cx(q) + M::cy(q) * M::cy(q) + M::cz(q) * M::cz(q));
            v[0] += a.m.rho_ref;
            v[4] += a.m.rho_ref * e_ref;
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] *= V;
    }
    // fixed-order tree: within each warp by shuffles, then the warps' sums in warp order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    constexpr int NW = BS / 32;
    if ((l & 31) == 0)
#pragma unroll
        for (int j = 0; j < 5; ++j) red[j][l >> 5] = v[j];
    __syncthreads();
    if (l < 5) {
        double s = red[l][0];
#pragma unroll
        for (int w = 1; w < NW; ++w) s += red[l][w];
        partial[bid * 5 + l] = s;
    }
}

template <class M, int ST, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ) k_ledger(const StepArgs a, double* partial) {
    ledger_block<M, ST, BX, BY, BZ>(a, blockIdx.x, partial);
}

static __global__ void __launch_bounds__(1024) k_ledger_final(const double* partial, long long n, double* out) {
    __shared__ double red[5][1024];
    const int l = threadIdx.x;
    double v[5] = {0, 0, 0, 0, 0};
    for (long long i = l; i < n; i += 1024)
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] += partial[i * 5 + j];
#pragma unroll
    for (int j = 0; j < 5; ++j) red[j][l] = v[j];
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (l < s) {
#pragma unroll
            for (int j = 0; j < 5; ++j) red[j][l] += red[j][l + s];
        }
        __syncthreads();
    }
    if (l < 5) out[l] = red[l][0];
}

// ------------------------------------------------------------------ state upload
// Pre-collision state as stored (f: Q x ncell, deviations f - w rho_ref for the deviation formats,
// then g: Q x ncell for the double distribution, then lambda: 8 x ncell, slot-indexed) into
// buffer 1, lambda into both buffers; absent and solid slots get zero populations.  The prestream
// pass then writes buffer 0.
template <class M, int ST, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ) k_load_state(const StepArgs a, int lev, const double* __restrict__ full) {
    using T = typename Store<ST>::T;
    constexpr int BS = BX * BY * BZ;
    const LevelDev& L = a.lv[lev];
    const long long b = blockIdx.x;
    const int l = threadIdx.x;
    const long long cell = b * BS + l;
    const long long n = L.ncell;
    const int type = (b == L.nb) ? (int)C_ABSENT : (L.bflag[b] == 1 ? (int)C_FLUID : (int)L.type[cell]);
    const bool zero = type == C_ABSENT || type == C_SOLID;
#pragma unroll 1
    for (int q = 0; q < M::Q; ++q) {
        const T ref = M::DEV ? ref_f<M, ST>(a.m, q) : T(0);
        const T fv = zero ? -ref : T(full[(long long)q * n + cell]);
        const T gv = (M::HAS_G && !zero) ? T(full[(long long)(M::Q + q) * n + cell]) : T(0);
        store_pop<M, ST, BS>(L, 1, cell, q, a.m, fv, gv);
        if (zero) store_pop<M, ST, BS>(L, 0, cell, q, a.m, fv, gv);
    }
    if constexpr (M::HAS_LAM) {
        if (b < L.nb) {
            const long long o = (long long)(M::HAS_G ? 2 * M::Q : M::Q) * n;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const double v = zero ? 0.0 : full[o + (long long)i * n + cell];
                L.lam[((long long)0 * 8 + i) * n + cell] = v;
                L.lam[((long long)1 * 8 + i) * n + cell] = v;
            }
        }
    }
}

// After a remesh (level lev >= 1, state just loaded): a coarse ghost at a concave corner lets
// its own streamed population stand in for children whose history leaves the finer level; those
// populations are set to (2^D v - sum of the other children) / (number of such children), v the
// ghost's carried state, so that its coalesced state is v and the ledger is kept exactly.
template <class M, int ST, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ) k_remesh_corners(const StepArgs a, int lev) {
    using T = typename Store<ST>::T;
    constexpr int BS = BX * BY * BZ;
    constexpr int NK = (M::D == 3) ? 8 : 4;
    const LevelDev& L = a.lv[lev];
    const LevelDev& F = a.lv[lev - 1];
    const long long b = blockIdx.x;
    const int l = threadIdx.x;
    const long long cell = b * BS + l;
    if (L.bflag[b] == 1 || L.type[cell] != C_CGHOST) return;
    const CellRecDev rec = L.recs[L.rec_id[cell]];
    if (!(rec.b & 1)) return;
#pragma unroll 1
    for (int q = 0; q < M::Q; ++q) {
        if (!(rec.mask >> q & 1ull)) continue;
        int cx = 0, cy = 0, cz = 0;
#pragma unroll
        for (int qq = 0; qq < M::Q; ++qq)
            if (qq == q) { cx = M::cx(qq); cy = M::cy(qq); cz = M::cz(qq); }
        const long long s = src_cell_g<BX, BY, BZ>(L.nbr, cell, cx, cy, cz);
        T vf, vg;
        load_pop<M, ST, BS>(L, 0, s, q, a.m, vf, vg);
        T rf = T(0), rg = T(0);
        int nb = 0;
#pragma unroll 1
        for (int k = 0; k < NK; ++k) {
            const long long ch = rec.a + (k & 1) + ((k >> 1) & 1) * BX + ((k >> 2) & 1) * BX * BY;
            if (history_leaves<M, BX, BY, BZ>(F, ch, cx, cy, cz)) {
                ++nb;
                continue;
            }
            T cf, cg;
            load_pop<M, ST, BS>(F, 0, src_cell_g<BX, BY, BZ>(F.nbr, ch, cx, cy, cz), q, a.m, cf, cg);
            rf += cf;
            rg += cg;
        }
        if (!nb) continue;
        store_pop<M, ST, BS>(L, 0, s, q, a.m, (T(NK) * vf - rf) / T(nb), (T(NK) * vg - rg) / T(nb));
    }
}

// ------------------------------------------------------------------ initialisation
// Pass 1: equilibrium E of the given fields into buffer 1 (and lambda into both lambda buffers).
template <class M, int ST, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ) k_init_eq(const StepArgs a, int lev, const double* rho_in,
                                                          const double* u_in, const double* T_in) {
    using T = typename Store<ST>::T;
    constexpr int BS = BX * BY * BZ;
    const LevelDev& L = a.lv[lev];
    const long long b = blockIdx.x;
    const int l = threadIdx.x;
    const long long cell = b * BS + l;
    // block nb (one past the last) is the zero-population block; absent and solid slots hold
    // zero populations in both buffers too, so that a plain gather reads a zero where the
    // pull has no source
    const int type = (b == L.nb) ? (int)C_ABSENT : (L.bflag[b] == 1 ? (int)C_FLUID : (int)L.type[cell]);
    if (type == C_ABSENT || type == C_SOLID) {
#pragma unroll 1
        for (int q = 0; q < M::Q; ++q) {
            const T z = M::DEV ? -ref_f<M, ST>(a.m, q) : T(0);
            store_pop<M, ST, BX * BY * BZ>(L, 0, cell, q, a.m, z, T(0));
            store_pop<M, ST, BX * BY * BZ>(L, 1, cell, q, a.m, z, T(0));
        }
        return;
    }
    const long long n = L.ncell;
    const T rho = T(rho_in[cell]);
    const T ux = T(u_in[cell]), uy = T(u_in[n + cell]), uz = T(M::D == 3 ? u_in[2 * n + cell] : 0.0);
    T feq[M::Q];
    if constexpr (!M::HAS_G) {
        if constexpr (hermite_weak<M>::value) M::template feq_dev<T>(rho, ux, uy, T(a.m.rho_ref), feq);
        else weak_feq_dev<M::D, T>(rho, ux, uy, uz, T(a.m.rho_ref), feq);
#pragma unroll
        for (int q = 0; q < M::Q; ++q)
            store_pop<M, ST, BX * BY * BZ>(L, 1, cell, a.aa ? M::Q - 1 - q : q, a.m, feq[q], T(0));
    } else {
        const T Tt = T(T_in[cell]);
        double lam[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int it, conv;
        if constexpr (M::HAS_LAM) M::init_guess((double)ux, (double)uy, (double)Tt, lam);
        ModelDev m = a.m;
        m.guess = 0;              // start from the polynomial guess computed above
        M::template feq<ST>(m, rho, ux, uy, Tt, lam, feq, &it, &conv);
        if (!conv) set_status(a.status, -6);
        const T gfac = T((2.0 * a.m.Cv - M::D) * (double)Tt);
#pragma unroll
        for (int q = 0; q < M::Q; ++q)
            store_pop<M, ST, BX * BY * BZ>(L, 1, cell, a.aa ? M::Q - 1 - q : q, a.m, feq[q], gfac * feq[q]);
        if constexpr (M::HAS_LAM) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                L.lam[((long long)0 * 8 + i) * n + cell] = lam[i];
                L.lam[((long long)1 * 8 + i) * n + cell] = lam[i];
            }
        }
    }
}

// Pass 2: stored_q(y) = E_q(y + xi_q), or E_qbar(y) where y's link qbar is blocked, so that the
// first gather reproduces E at every cell (the stored state is post-collision populations).
template <class M, int ST, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ) k_init_prestream(const StepArgs a, int lev) {
    using S = typename Store<ST>::S;
    constexpr int BS = BX * BY * BZ;
    __shared__ int nbr_s[27];
    const LevelDev& L = a.lv[lev];
    const long long b = blockIdx.x;
    const int l = threadIdx.x;
    if (l < 27) nbr_s[l] = L.nbr[b * 27 + l];
    __syncthreads();
    const long long cell = b * BS + l;
    const int type = L.bflag[b] == 1 ? (int)C_FLUID : (int)L.type[cell];
    if (type == C_ABSENT || type == C_SOLID) return;
    unsigned long long bmask = 0ull;
    bool walls = false;
    if (L.bflag[b] != 1 && type == C_FLUID) {
        const int r = L.rec_id[cell];
        if (r >= 0) {
            bmask = L.recs[r].mask;
            walls = (L.recs[r].b & 2) != 0;
        }
    }
    const int lx = l % BX, ly = (l / BX) % BY, lz = l / (BX * BY);
    const S* Ef = (const S*)L.f[1];
    const S* Eg = (const S*)L.g[1];
    S* Of = (S*)L.f[0];
    S* Og = (S*)L.g[0];
#pragma unroll
    for (int q = 0; q < M::Q; ++q) {
        const int qb = M::Q - 1 - q;
        long long src;
        int qs;
        if constexpr (!M::HAS_G) {
            if (walls && (bmask & (1ull << qb))) {
                // a link bounced at a moving wall: the first gather adds the wall term back
                using T = typename Store<ST>::T;
                T e, dummy;
                load_pop<M, ST, BS>(L, 1, cell, qb, a.m, e, dummy);
                store_pop<M, ST, BS>(L, 0, cell, q, a.m, e - T(wall_term<M, BX, BY, BZ>(a.m, L, b, l, qb)), T(0));
                continue;
            }
        }
        if (bmask & (1ull << qb)) {
            src = cell;
            qs = qb;
        } else {
            src = src_cell<BX, BY, BZ>(nbr_s, b, lx, ly, lz, -M::cx(q), -M::cy(q), -M::cz(q));
            qs = q;
            if (src >= 0) {
                const int st = L.type[src];
                if (st == C_ABSENT || st == C_SOLID) src = -1;
            }
        }
        S vf, vg;
        if (src >= 0) {
            vf = Ef[pidx<BS, M::Q>(src, qs)];
            if constexpr (M::HAS_G) vg = Eg[pidx<BS, M::Q>(src, qs)];
        } else {
            // zero population: -1 in the binary16 format, -ref for the other deviation formats
            vf = S(ST == ST_F16DEV ? -1.0f : (M::DEV ? -ref_f<M, ST>(a.m, q) : 0.0f));
            vg = S(ST == ST_F16DEV ? -1.0f : 0.0f);
        }
        Of[pidx<BS, M::Q>(cell, q)] = vf;
        if constexpr (M::HAS_G) Og[pidx<BS, M::Q>(cell, q)] = vg;
    }
}

// ------------------------------------------------------------------ host launchers
template <class M, int ST, int BX, int BY, int BZ>
struct Launch {
    // DIRECT: the simple blocks gather straight from global memory also where a staged kernel exists
    template <int MINB_F, int MINB_G, bool DIRECT = false>
    static void step(const StepArgs& a, long long n_fast, long long n_gen, cudaStream_t s_fast, cudaStream_t s_gen) {
        // interior sweep first; the few, latency-bound general blocks fill in as its blocks retire
        if (n_fast) {
            if constexpr (staged_f16<M, ST, BX, BY, BZ>::value && !DIRECT)
                k_step_staged<M, ST, BX, BY, BZ, MINB_F, staged_nb(MINB_F)>
                    <<<(unsigned)((n_fast + staged_nb(MINB_F) - 1) / staged_nb(MINB_F)), BX * BY * BZ / 2, 0, s_fast>>>(a);
            else
                k_step<M, ST, BX, BY, BZ, true, MINB_F><<<(unsigned)n_fast, BX * BY * BZ, 0, s_fast>>>(a);
        }
        if (n_gen) k_step<M, ST, BX, BY, BZ, false, MINB_G><<<(unsigned)n_gen, BX * BY * BZ, 0, s_gen>>>(a);
    }
    template <int MINB_F, int MINB_G>
    static void batch(const StepArgs* args, const long long* off_fast, const long long* off_gen, int n,
                      long long n_fast, long long n_gen, cudaStream_t s_fast, cudaStream_t s_gen) {
        if (n_gen) k_step_batch<M, ST, BX, BY, BZ, false, MINB_G><<<(unsigned)n_gen, BX * BY * BZ, 0, s_gen>>>(args, off_gen, n);
        if (n_fast) k_step_batch<M, ST, BX, BY, BZ, true, MINB_F><<<(unsigned)n_fast, BX * BY * BZ, 0, s_fast>>>(args, off_fast, n);
    }
    static void read(const StepArgs& a, int lev, int which, double* out, cudaStream_t s) {
        if (a.lv[lev].nb) k_read<M, ST, BX, BY, BZ><<<(unsigned)a.lv[lev].nb, BX * BY * BZ, 0, s>>>(a, lev, which, out);
    }
    static void load_state(const StepArgs& a, int lev, const double* full, cudaStream_t s) {
        if (!a.lv[lev].nb) return;
        k_load_state<M, ST, BX, BY, BZ><<<(unsigned)a.lv[lev].nb + 1, BX * BY * BZ, 0, s>>>(a, lev, full);
        k_init_prestream<M, ST, BX, BY, BZ><<<(unsigned)a.lv[lev].nb, BX * BY * BZ, 0, s>>>(a, lev);
    }
    static void remesh_corners(const StepArgs& a, int lev, cudaStream_t s) {
        if (lev >= 1 && a.lv[lev].nb) k_remesh_corners<M, ST, BX, BY, BZ><<<(unsigned)a.lv[lev].nb, BX * BY * BZ, 0, s>>>(a, lev);
    }
    static void ledger(const StepArgs& a, long long nblocks, double* partial, double* out, cudaStream_t s) {
        if (nblocks) k_ledger<M, ST, BX, BY, BZ><<<(unsigned)nblocks, BX * BY * BZ, 0, s>>>(a, partial);
        k_ledger_final<<<1, 1024, 0, s>>>(partial, nblocks, out);
    }
    static void init(const StepArgs& a, int lev, const double* r, const double* u, const double* t, cudaStream_t s) {
        if (!a.lv[lev].nb) return;
        k_init_eq<M, ST, BX, BY, BZ><<<(unsigned)a.lv[lev].nb + 1, BX * BY * BZ, 0, s>>>(a, lev, r, u, t);
        // AA streaming starts in layout L1 (one buffer, each cell's own slots reversed)
        if (!a.aa) k_init_prestream<M, ST, BX, BY, BZ><<<(unsigned)a.lv[lev].nb, BX * BY * BZ, 0, s>>>(a, lev);
    }
    // one AA iteration of the single level; its parity is a.rd[0] (odd: L0 -> L1)
    static void aa(const StepArgs& a, cudaStream_t s) {
        if constexpr (aa_capable<M>::value) {
            const unsigned nb = (unsigned)a.lv[0].nb;
            if (!nb) return;
            if (a.rd[0]) k_step_aa<M, ST, BX, BY, BZ, true><<<nb, BX * BY * BZ, 0, s>>>(a);
            else k_step_aa<M, ST, BX, BY, BZ, false><<<nb, BX * BY * BZ, 0, s>>>(a);
        }
    }
};

template <class M, int ST, int BX, int BY, int BZ>
KernelSet make_set() {
    KernelSet k;
    using LS = Launch<M, ST, BX, BY, BZ>;
    k.step = &LS::template step<0, 0>;
    k.variant[0] = &LS::template step<0, 0>;
    k.variant_minb[0] = 0;
    k.n_variants = 1;
    if constexpr (M::BATCH) k.batch[0] = &LS::template batch<0, 0>;
    if constexpr (M::TUNE && ST != ST_F64) {       // occupancy targets tried by the autotuner
        // M::TUNE_V: (interior kernel, general kernel) resident 128-thread blocks, 10 * F + G
        constexpr int V0 = M::TUNE_V[0], V1 = M::TUNE_V[1], V2 = M::TUNE_V[2];
        k.variant[1] = &LS::template step<V0 / 10, V0 % 10>;
        k.variant[2] = &LS::template step<V1 / 10, V1 % 10>;
        k.variant[3] = &LS::template step<V2 / 10, V2 % 10>;
        if constexpr (M::BATCH) {
            k.batch[1] = &LS::template batch<V0 / 10, V0 % 10>;
            k.batch[2] = &LS::template batch<V1 / 10, V1 % 10>;
            k.batch[3] = &LS::template batch<V2 / 10, V2 % 10>;
        }
        k.variant_minb[1] = V0;
        k.variant_minb[2] = V1;
        k.variant_minb[3] = V2;
        k.n_variants = 4;
        if constexpr (staged_f16<M, ST, BX, BY, BZ>::value) {   // the direct-gather forms, codes 100 + target
            k.variant[4] = &LS::template step<0, 0, true>;
            k.variant[5] = &LS::template step<V0 / 10, V0 % 10, true>;
            k.variant[6] = &LS::template step<V1 / 10, V1 % 10, true>;
            k.variant[7] = &LS::template step<V2 / 10, V2 % 10, true>;
            k.variant_minb[4] = 100;
            k.variant_minb[5] = 100 + V0;
            k.variant_minb[6] = 100 + V1;
            k.variant_minb[7] = 100 + V2;
            k.n_variants = 8;
        }
    }
    k.read = &Launch<M, ST, BX, BY, BZ>::read;
    k.ledger = &Launch<M, ST, BX, BY, BZ>::ledger;
    k.init = &Launch<M, ST, BX, BY, BZ>::init;
    k.load_state = &Launch<M, ST, BX, BY, BZ>::load_state;
    k.remesh_corners = &Launch<M, ST, BX, BY, BZ>::remesh_corners;
    if constexpr (aa_capable<M>::value) k.aa = &Launch<M, ST, BX, BY, BZ>::aa;
    k.step_kernel = (const void*)&k_step<M, ST, BX, BY, BZ, true, 0>;   // for occupancy queries
    k.block_threads = BX * BY * BZ;
    return k;
}

template <class M, int BX, int BY, int BZ>
bool pick_storage(int storage, KernelSet& out) {
    switch (storage) {
        case ST_F64: out = make_set<M, ST_F64, BX, BY, BZ>(); return true;
        case ST_F32: out = make_set<M, ST_F32, BX, BY, BZ>(); return true;
        case ST_F16DEV:
            if constexpr (weak_var<M>::value == 0) {       // the collision variants: FP64 and FP32 only
                out = make_set<M, ST_F16DEV, BX, BY, BZ>();
                return true;
            }
            return false;
    }
    return false;
}

}  // namespace lbm
