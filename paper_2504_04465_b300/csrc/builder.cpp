// Host grid builder: see builder.h.
//
// Cell sets per level (Sec. 3.2, Fig. rohde_highorder): with Region_i the union of the level-i
// boxes (the whole domain for the coarsest level),
//   bulk_i   = cells of Region_i not covered by Region_{i-1}
//   cghost_i = cells covered by Region_{i-1} within `reach` (Chebyshev, level-i units) of bulk_i
//   fghost_i = children of cghost_{i+1}  (2*reach fine layers)
// A coarse-ghost population is supplied by coalescence unless it was streamed from a coarse
// bulk or boundary cell (the rest population always stays); with that rule the coupling is
// exactly conservative, including at patch corners where diagonal links cut through the fine
// bulk.  Wall faces have no boundary layer: a link whose source leaves the domain through wall
// faces only bounces back (record mask bit, b bit 1 for the moving-wall term).  At concave
// corners of the finer region a child's two-step streaming history can leave
// the finer level; such a child enters the coalescence with the ghost's own streamed
// population, which keeps the coupling conservative there too (record flag b bit 0).  Boundary layers are the `reach` outer layers on non-periodic faces (Appendix A.3); a
// boundary cell's partner is the cell obtained by clamping its coordinates into the interior.
// Blocks whose only special cells are fine ghosts, absent slots and Neumann boundary cells with
// their partner in the block are streaming blocks of the interior kernels.
// A link is blocked by a solid when any cell met on the lattice segment is solid, taking both
// roundings where the segment passes between cells.
#include "builder.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <omp.h>

namespace lbm {
namespace {

struct Geo {
    const GridInput& in;
    LatticeDesc lat;
    int D = 2, L = 1, R = 1;
    int B[3] = {1, 1, 1};
    int64_t shape[16][3];
    bool periodic[3] = {true, true, true};

    explicit Geo(const GridInput& g) : in(g) {}

    // box expressed in level-`i` cell units (alignment checked earlier)
    bool in_box(const BoxSpec& b, int i, const int64_t* c) const {
        for (int d = 0; d < D; ++d) {
            int64_t lo = b.lo[d] >> i, hi = b.hi[d] >> i;
            if (c[d] < lo || c[d] >= hi) return false;
        }
        return true;
    }
    // regions as dense per-level masks (from a level map), else from the boxes
    std::vector<std::vector<uint8_t>> rmask;
    int64_t lidx(int i, const int64_t* c) const { return (c[2] * shape[i][1] + c[1]) * shape[i][0] + c[0]; }
    bool in_region(int i, const int64_t* c) const {
        if (i >= L - 1) return true;
        if (!rmask.empty()) return rmask[i][lidx(i, c)] != 0;
        for (auto& b : in.boxes)
            if (b.level == i && in_box(b, i, c)) return true;
        return false;
    }
    bool finer(int i, const int64_t* c) const {
        if (i == 0) return false;
        if (!rmask.empty()) {
            const int64_t ch[3] = {2 * c[0], D > 1 ? 2 * c[1] : c[1], D > 2 ? 2 * c[2] : c[2]};
            return rmask[i - 1][lidx(i - 1, ch)] != 0;
        }
        for (auto& b : in.boxes)
            if (b.level == i - 1 && in_box(b, i, c)) return true;
        return false;
    }
    bool bulk(int i, const int64_t* c) const { return in_region(i, c) && !finer(i, c); }
    // wrap into the domain; false if outside a non-periodic face
    bool wrap(int i, const int64_t* c, int64_t* o) const {
        for (int d = 0; d < 3; ++d) o[d] = c[d];
        for (int d = 0; d < D; ++d) {
            int64_t n = shape[i][d];
            if (o[d] < 0 || o[d] >= n) {
                if (!periodic[d]) return false;
                o[d] = ((o[d] % n) + n) % n;
            }
        }
        return true;
    }
    bool cghost(int i, const int64_t* c) const {
        if (!finer(i, c)) return false;
        int64_t o[3], w[3];
        int rz = D == 3 ? R : 0;
        for (int dz = -rz; dz <= rz; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    o[0] = c[0] + dx; o[1] = c[1] + dy; o[2] = c[2] + dz;
                    if (wrap(i, o, w) && bulk(i, w)) return true;
                }
        return false;
    }
    bool is_cell(int i, const int64_t* c) const { return bulk(i, c) || cghost(i, c); }
    // within the lattice reach of a wall face
    bool near_wall(int i, const int64_t* c) const {
        for (int d = 0; d < D; ++d) {
            if (periodic[d]) continue;
            if (in.faces[2 * d].kind == BCK_WALL && c[d] < R) return true;
            if (in.faces[2 * d + 1].kind == BCK_WALL && c[d] >= shape[i][d] - R) return true;
        }
        return false;
    }
    // the pull source c - xi leaves the domain through wall faces only (periodic axes wrap)
    bool wall_link(int i, const int64_t* c, const int* xi) const {
        int walls = 0;
        for (int d = 0; d < D; ++d) {
            if (periodic[d]) continue;
            const int64_t s = c[d] - xi[d];
            int f = -1;
            if (s < 0) f = 2 * d;
            else if (s >= shape[i][d]) f = 2 * d + 1;
            if (f < 0) continue;
            if (in.faces[f].kind != BCK_WALL) return false;
            ++walls;
        }
        return walls > 0;
    }
    bool fghost(int i, const int64_t* c) const {
        if (i + 1 >= L) return false;
        int64_t p[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
        return cghost(i + 1, p);
    }
    bool solid(int i, const int64_t* c) const {
        if (i != 0) return false;
        double x[3] = {c[0] + 0.5, c[1] + 0.5, c[2] + 0.5};
        for (auto& s : in.solids) {
            if (s.kind == 1) {
                double r2 = 0;
                for (int d = 0; d < D; ++d) r2 += (x[d] - s.p[d]) * (x[d] - s.p[d]);
                if (r2 < s.p[3] * s.p[3]) return true;
            } else if (s.kind == 2) {
                // symmetric NACA 4-digit thickness (closed trailing edge), zero angle of attack
                double ch = s.p[0], x0 = s.p[1], y0 = s.p[2], t = s.p[3];
                double xr = (x[0] - x0) / ch;
                if (xr < 0.0 || xr > 1.0) continue;
                double yt = 5.0 * t * ch * (0.2969 * std::sqrt(xr) - 0.1260 * xr - 0.3516 * xr * xr +
                                             0.2843 * xr * xr * xr - 0.1036 * xr * xr * xr * xr);
                if (std::fabs(x[1] - y0) < yt) return true;
            }
        }
        return false;
    }
    void solid_bbox(const ShapeSpec& s, double lo[3], double hi[3]) const {
        for (int d = 0; d < 3; ++d) { lo[d] = -1e30; hi[d] = 1e30; }
        if (s.kind == 1) {
            for (int d = 0; d < D; ++d) { lo[d] = s.p[d] - s.p[3] - 1; hi[d] = s.p[d] + s.p[3] + 1; }
        } else {
            lo[0] = s.p[1] - 1; hi[0] = s.p[1] + s.p[0] + 1;
            lo[1] = s.p[2] - 0.07 * s.p[0] - 1; hi[1] = s.p[2] + 0.07 * s.p[0] + 1;
        }
    }
    int bc_face(int i, const int64_t* c) const {
        // highest-priority face among the faces whose reach layer contains c:
        // any Dirichlet face over Neumann; among equals the first face
        int best = -1;
        for (int d = 0; d < D; ++d) {
            if (periodic[d]) continue;
            for (int side = 0; side < 2; ++side) {
                bool in_layer = side == 0 ? c[d] < R : c[d] >= shape[i][d] - R;
                if (!in_layer) continue;
                int f = 2 * d + side;
                if (in.faces[f].kind == BCK_WALL) continue;      // walls have no boundary layer
                if (best < 0) { best = f; continue; }
                int kb = in.faces[best].kind, kf = in.faces[f].kind;
                if (kb == BCK_NEUMANN && kf != BCK_NEUMANN) best = f;
            }
        }
        return best;
    }
};

uint64_t morton(int64_t x, int64_t y, int64_t z) {
    auto spread = [](uint64_t v) {
        uint64_t r = 0;
        for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
        return r;
    };
    return spread(x) | (spread(y) << 1) | (spread(z) << 2);
}

// cells met on the segment from x to x - xi: offsets o such that x - o is checked
void segment_offsets(const int* xi, int D, std::vector<std::array<int, 3>>& out) {
    out.clear();
    int n = 0;
    for (int d = 0; d < D; ++d) n = std::max(n, std::abs(xi[d]));
    for (int m = 1; m <= n; ++m) {
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) {
            int num = m * xi[d];
            int fl = (num >= 0) ? num / n : -((-num + n - 1) / n);
            int cl = (num >= 0) ? (num + n - 1) / n : -((-num) / n);
            lo[d] = fl; hi[d] = cl;
        }
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c) {
                    std::array<int, 3> o{a, b, c};
                    if (std::find(out.begin(), out.end(), o) == out.end()) out.push_back(o);
                }
    }
}

}  // namespace

std::string build_grid(const GridInput& in, BuiltGrid& out) {
    Geo g(in);
    g.lat = lattice_desc(in.lattice);
    if (g.lat.Q == 0) return "unknown lattice";
    g.D = in.dim;
    g.L = in.n_levels;
    g.R = g.lat.R;
    if (g.D != g.lat.D) return "lattice dimension differs from the context dimension";
    if (g.L < 1 || g.L > 8) return "n_levels must be in [1, 8]";
    for (int d = 0; d < 3; ++d) g.B[d] = (d < g.D) ? in.block[d] : 1;
    for (int d = 0; d < g.D; ++d) {
        if (g.B[d] < 2 || (g.B[d] & 1) || g.B[d] < g.R) return "block extents must be even and >= the lattice reach";
        g.periodic[d] = in.faces[2 * d].kind == BCK_PERIODIC;
        if ((in.faces[2 * d + 1].kind == BCK_PERIODIC) != g.periodic[d]) return "both faces of an axis must be periodic or neither";
    }
    for (int d = g.D; d < 3; ++d) g.periodic[d] = true;
    for (int i = 0; i < g.L; ++i)
        for (int d = 0; d < 3; ++d) {
            int64_t e = (d < g.D) ? in.extent[d] : 1;
            if (d < g.D && (e <= 0 || e % (int64_t(1) << i))) return "extent not divisible by 2^(n_levels-1)";
            g.shape[i][d] = (d < g.D) ? (e >> i) : 1;
            if (d < g.D && g.periodic[d] && g.shape[i][d] % g.B[d]) return "periodic extent of a level not a multiple of the block";
        }
    for (auto& b : in.boxes) {
        if (b.level < 0 || b.level > g.L - 2) return "box level out of range";
        int64_t al = int64_t(2) << b.level;
        for (int d = 0; d < g.D; ++d) {
            if (b.lo[d] % al || b.hi[d] % al) return "box not aligned to 2^(level+1)";
            if (b.lo[d] < 0 || b.hi[d] > in.extent[d] || b.lo[d] >= b.hi[d]) return "box outside the domain or empty";
        }
        if (b.level + 1 < g.L - 1) {
            bool ok = false;
            for (auto& c : in.boxes) {
                if (c.level != b.level + 1) continue;
                bool inside = true;
                for (int d = 0; d < g.D; ++d) inside &= c.lo[d] <= b.lo[d] && b.hi[d] <= c.hi[d];
                ok |= inside;
            }
            if (!ok) return "box not nested in a box of the next coarser level";
        }
    }
    for (auto& s : in.solids)
        if (s.kind != 1 && s.kind != 2) return "unknown solid kind";
    if (!in.level_map.empty()) {
        if (!in.boxes.empty()) return "give refinement boxes or a level map, not both";
        int64_t n0 = g.shape[0][0] * g.shape[0][1] * g.shape[0][2];
        if ((int64_t)in.level_map.size() != n0) return "level map size differs from the finest extent";
        // min over the finest cells under each level-j cell, then region_i = cells whose parent
        // holds a finest cell wanting level i or finer (aligned to parents by construction)
        std::vector<uint8_t> minmap = in.level_map;
        for (auto v : minmap)
            if (v >= g.L) return "level map entry beyond the coarsest level";
        std::vector<std::vector<uint8_t>> mins(g.L);
        mins[0] = minmap;
        for (int j = 1; j < g.L; ++j) {
            const int64_t* sj = g.shape[j];
            std::vector<uint8_t> m(sj[0] * sj[1] * sj[2], 255);
            const int64_t* sp = g.shape[j - 1];
            for (int64_t z = 0; z < sp[2]; ++z)
                for (int64_t y = 0; y < sp[1]; ++y)
                    for (int64_t x = 0; x < sp[0]; ++x) {
                        const int64_t pz = g.D > 2 ? z >> 1 : z, py = y >> 1, px = x >> 1;
                        uint8_t& t = m[(pz * sj[1] + py) * sj[0] + px];
                        t = std::min(t, mins[j - 1][(z * sp[1] + y) * sp[0] + x]);
                    }
            mins[j] = std::move(m);
        }
        g.rmask.resize(g.L - 1);
        for (int i = 0; i + 1 < g.L; ++i) {
            const int64_t* si = g.shape[i];
            const int64_t* sp = g.shape[i + 1];
            g.rmask[i].assign(si[0] * si[1] * si[2], 0);
            for (int64_t z = 0; z < si[2]; ++z)
                for (int64_t y = 0; y < si[1]; ++y)
                    for (int64_t x = 0; x < si[0]; ++x) {
                        const int64_t pz = g.D > 2 ? z >> 1 : z;
                        g.rmask[i][(z * si[1] + y) * si[0] + x] = mins[i + 1][(pz * sp[1] + (y >> 1)) * sp[0] + (x >> 1)] <= i;
                    }
        }
    }

    out = BuiltGrid{};
    out.dim = g.D; out.n_levels = g.L; out.lat = g.lat;
    for (int d = 0; d < 3; ++d) { out.block[d] = g.B[d]; out.periodic[d] = g.periodic[d]; }
    const int BS = g.B[0] * g.B[1] * g.B[2];
    out.BS = BS;
    const int M = 3 * g.R + 2;          // margin of the plain-block test

    for (int i = 0; i < g.L; ++i) {
        BuiltLevel lv;
        lv.level = i;
        for (int d = 0; d < 3; ++d) {
            lv.shape[d] = g.shape[i][d];
            lv.bgrid[d] = (lv.shape[d] + g.B[d] - 1) / g.B[d];
        }
        // candidate blocks: intersecting a box of level i (all blocks for the coarsest level)
        std::vector<int64_t> cand;
        const int64_t nbg = lv.bgrid[0] * lv.bgrid[1] * lv.bgrid[2];
        std::vector<uint8_t> mark(nbg, 0);
        if (i == g.L - 1) {
            std::fill(mark.begin(), mark.end(), 1);
        } else if (!g.rmask.empty()) {
            for (int64_t z = 0; z < lv.shape[2]; ++z)
                for (int64_t y = 0; y < lv.shape[1]; ++y)
                    for (int64_t x = 0; x < lv.shape[0]; ++x)
                        if (g.rmask[i][(z * lv.shape[1] + y) * lv.shape[0] + x])
                            mark[((z / g.B[2]) * lv.bgrid[1] + y / g.B[1]) * lv.bgrid[0] + x / g.B[0]] = 1;
        } else {
            for (auto& b : in.boxes) {
                if (b.level != i) continue;
                int64_t lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
                for (int d = 0; d < g.D; ++d) {
                    lo[d] = (b.lo[d] >> i) / g.B[d];
                    hi[d] = ((b.hi[d] >> i) + g.B[d] - 1) / g.B[d];
                }
                for (int64_t z = lo[2]; z < hi[2]; ++z)
                    for (int64_t y = lo[1]; y < hi[1]; ++y)
                        for (int64_t x = lo[0]; x < hi[0]; ++x)
                            mark[(z * lv.bgrid[1] + y) * lv.bgrid[0] + x] = 1;
            }
        }
        for (int64_t k = 0; k < nbg; ++k)
            if (mark[k]) cand.push_back(k);
        const int64_t nc = (int64_t)cand.size();
        std::vector<uint8_t> ctype(nc * BS, C_ABSENT);
        std::vector<uint8_t> plain(nc, 0);
        std::vector<uint8_t> live(nc, 0);
        std::vector<std::string> errs(omp_get_max_threads());

#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t k = 0; k < nc; ++k) {
            int64_t bk = cand[k];
            int64_t bc[3] = {bk % lv.bgrid[0], (bk / lv.bgrid[0]) % lv.bgrid[1], bk / (lv.bgrid[0] * lv.bgrid[1])};
            int64_t c0[3], c1[3];
            for (int d = 0; d < 3; ++d) { c0[d] = bc[d] * g.B[d]; c1[d] = c0[d] + g.B[d]; }
            // plain test: block expanded by M inside the domain, inside one level-i box, away
            // from every finer box and every solid -> every cell and every source is bulk fluid
            bool pl = true;
            int64_t e0[3], e1[3];
            for (int d = 0; d < g.D; ++d) {
                e0[d] = c0[d] - M; e1[d] = c1[d] + M;
                if (e0[d] < 0 || e1[d] > lv.shape[d]) pl = false;
            }
            for (int d = g.D; d < 3; ++d) { e0[d] = 0; e1[d] = 1; }
            if (pl && !g.rmask.empty()) {
                // every cell of the expanded block in region i and none covered by region i-1
                for (int64_t z = e0[2]; z < e1[2] && pl; ++z)
                    for (int64_t y = e0[1]; y < e1[1] && pl; ++y)
                        for (int64_t x = e0[0]; x < e1[0] && pl; ++x) {
                            const int64_t cc[3] = {x, y, z};
                            if (!g.in_region(i, cc) || g.finer(i, cc)) pl = false;
                        }
            } else if (pl && i < g.L - 1) {
                bool inside = false;
                for (auto& b : in.boxes) {
                    if (b.level != i) continue;
                    bool ok = true;
                    for (int d = 0; d < g.D; ++d) ok &= (b.lo[d] >> i) <= e0[d] && e1[d] <= (b.hi[d] >> i);
                    inside |= ok;
                }
                pl = inside;
            }
            if (pl && i >= 1 && g.rmask.empty()) {
                for (auto& b : in.boxes) {
                    if (b.level != i - 1) continue;
                    bool overlap = true;
                    for (int d = 0; d < g.D; ++d) overlap &= (b.lo[d] >> i) < e1[d] && e0[d] < (b.hi[d] >> i);
                    if (overlap) { pl = false; break; }
                }
            }
            if (pl && i == 0) {
                for (auto& s : in.solids) {
                    double lo[3], hi[3];
                    g.solid_bbox(s, lo, hi);
                    bool overlap = true;
                    for (int d = 0; d < g.D; ++d) overlap &= lo[d] < e1[d] && e0[d] < hi[d];
                    if (overlap) { pl = false; break; }
                }
            }
            if (pl) {
                std::fill(&ctype[k * BS], &ctype[k * BS] + BS, (uint8_t)C_FLUID);
                plain[k] = 1;
                live[k] = 1;
                continue;
            }
            std::string& e = errs[omp_get_thread_num()];
            bool any = false;
            for (int lz = 0; lz < g.B[2]; ++lz)
                for (int ly = 0; ly < g.B[1]; ++ly)
                    for (int lx = 0; lx < g.B[0]; ++lx) {
                        int64_t c[3] = {c0[0] + lx, c0[1] + ly, c0[2] + lz};
                        bool inside = true;
                        for (int d = 0; d < g.D; ++d) inside &= c[d] < lv.shape[d];
                        uint8_t t = C_ABSENT;
                        if (inside && g.is_cell(i, c)) {
                            bool cg = g.cghost(i, c);
                            bool fg = g.fghost(i, c);
                            bool so = g.solid(i, c);
                            int bf = g.bc_face(i, c);
                            if (cg && fg) e = "a cell is both a coarse and a fine ghost (levels too close)";
                            if (fg && !g.bulk(i, c)) e = "fine ghosts overlap another ghost layer";
                            if (so && (cg || fg)) e = "solid inside a ghost layer";
                            if (bf >= 0 && (cg || fg)) e = "boundary layer overlaps a ghost layer";
                            if ((cg || fg) && g.near_wall(i, c)) e = "ghost layer within the reach of a wall face";
                            if (cg) t = C_CGHOST;
                            else if (fg) t = C_FGHOST;
                            else if (so) t = C_SOLID;
                            else if (bf >= 0) t = C_BC;
                            else t = C_FLUID;
                            any = true;
                        }
                        ctype[k * BS + (lz * g.B[1] + ly) * g.B[0] + lx] = t;
                    }
            live[k] = any;
        }
        for (auto& e : errs)
            if (!e.empty()) return e + " (level " + std::to_string(i) + ")";
        // keep live blocks, Morton order
        std::vector<int64_t> keep;
        for (int64_t k = 0; k < nc; ++k)
            if (live[k]) keep.push_back(k);
        auto code = [&](int64_t k) {
            int64_t bk = cand[k];
            return morton(bk % lv.bgrid[0], (bk / lv.bgrid[0]) % lv.bgrid[1], bk / (lv.bgrid[0] * lv.bgrid[1]));
        };
        std::sort(keep.begin(), keep.end(), [&](int64_t a, int64_t b) { return code(a) < code(b); });
        lv.nb = (int64_t)keep.size();
        if ((lv.nb + 1) * (int64_t)BS > INT32_MAX) return "level too large for 32-bit cell indices";
        lv.bxyz.resize(lv.nb * 3);
        lv.type.resize(lv.nb * BS);
        lv.bflag.assign(lv.nb, 0);
        lv.bindex.assign(nbg, -1);
        for (int64_t b = 0; b < lv.nb; ++b) {
            int64_t k = keep[b], bk = cand[k];
            lv.bxyz[3 * b + 0] = int32_t(bk % lv.bgrid[0]);
            lv.bxyz[3 * b + 1] = int32_t((bk / lv.bgrid[0]) % lv.bgrid[1]);
            lv.bxyz[3 * b + 2] = int32_t(bk / (lv.bgrid[0] * lv.bgrid[1]));
            lv.bindex[bk] = (int32_t)b;
            std::memcpy(&lv.type[b * BS], &ctype[k * BS], BS);
            lv.bflag[b] = plain[k];
        }
        out.levels.push_back(std::move(lv));
    }

    // ---------------------------------------------------------------- links and records
    auto locate = [&](int i, const int64_t* c, int64_t& cell) -> uint8_t {
        const BuiltLevel& lv = out.levels[i];
        int64_t w[3];
        if (!g.wrap(i, c, w)) { cell = -1; return C_ABSENT; }
        int64_t bc[3], l[3];
        for (int d = 0; d < 3; ++d) { bc[d] = w[d] / g.B[d]; l[d] = w[d] % g.B[d]; }
        int64_t bk = (bc[2] * lv.bgrid[1] + bc[1]) * lv.bgrid[0] + bc[0];
        int32_t b = lv.bindex[bk];
        if (b < 0) { cell = -1; return C_ABSENT; }
        cell = int64_t(b) * BS + (l[2] * g.B[1] + l[1]) * g.B[0] + l[0];
        return lv.type[cell];
    };
    const int Q = g.lat.Q;
    std::vector<std::vector<std::array<int, 3>>> segs(Q);
    for (int q = 0; q < Q; ++q) segment_offsets(g.lat.xi[q], g.D, segs[q]);
    int rest = -1;
    for (int q = 0; q < Q; ++q)
        if (!g.lat.xi[q][0] && !g.lat.xi[q][1] && !g.lat.xi[q][2]) rest = q;

    for (int i = 0; i < g.L; ++i) {
        BuiltLevel& lv = out.levels[i];
        lv.nbr.assign(lv.nb * 27, -1);
        for (int64_t b = 0; b < lv.nb; ++b)
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (g.D == 2 && dz) continue;
                        int64_t nb[3] = {lv.bxyz[3 * b] + dx, lv.bxyz[3 * b + 1] + dy, lv.bxyz[3 * b + 2] + dz};
                        bool ok = true;
                        for (int d = 0; d < g.D; ++d) {
                            if (nb[d] < 0 || nb[d] >= lv.bgrid[d]) {
                                if (!g.periodic[d]) ok = false;
                                nb[d] = ((nb[d] % lv.bgrid[d]) + lv.bgrid[d]) % lv.bgrid[d];
                            }
                        }
                        if (!ok) continue;
                        lv.nbr[b * 27 + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] =
                            lv.bindex[(nb[2] * lv.bgrid[1] + nb[1]) * lv.bgrid[0] + nb[0]];
                    }
        lv.rec_id.assign(lv.nb * BS, -1);
        std::vector<std::vector<std::pair<int64_t, CellRec>>> trec(omp_get_max_threads());
        std::vector<std::string> errs(omp_get_max_threads());
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t b = 0; b < lv.nb; ++b) {
            if (lv.bflag[b]) continue;
            int tid = omp_get_thread_num();
            bool simple = true;
            // only record-free fluid cells, fine ghosts, absent slots and Neumann boundary cells
            // whose partner lies in the block (the interior kernels pull those at the partner)
            bool stream = true, neumann = false;
            for (int l = 0; l < BS; ++l) {
                int64_t cell = b * BS + l;
                uint8_t t = lv.type[cell];
                if (t != C_FLUID) simple = false;
                if (!(t == C_FLUID || t == C_FGHOST || t == C_ABSENT || t == C_BC)) stream = false;
                if (t == C_ABSENT || t == C_SOLID) continue;
                int lx = l % g.B[0], ly = (l / g.B[0]) % g.B[1], lz = l / (g.B[0] * g.B[1]);
                int64_t c[3] = {int64_t(lv.bxyz[3 * b]) * g.B[0] + lx, int64_t(lv.bxyz[3 * b + 1]) * g.B[1] + ly,
                                int64_t(lv.bxyz[3 * b + 2]) * g.B[2] + lz};
                CellRec r{0, -1, 0};
                bool need = false;
                if (t == C_FLUID || t == C_BC) {
                    for (int q = 0; q < Q; ++q) {
                        if (q == rest) continue;
                        int64_t s[3] = {c[0] - g.lat.xi[q][0], c[1] - g.lat.xi[q][1], c[2] - g.lat.xi[q][2]};
                        int64_t sc;
                        uint8_t st = locate(i, s, sc);
                        bool blocked = false;
                        if (i == 0) {
                            for (auto& o : segs[q]) {
                                int64_t p[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
                                int64_t pc;
                                if (locate(i, p, pc) == C_SOLID) { blocked = true; break; }
                            }
                        }
                        if (!blocked && st == C_ABSENT && g.wall_link(i, c, g.lat.xi[q])) {
                            // halfway bounce-back at a wall face (record b bit 1: the kernels add
                            // Ladd's moving-wall term to such links)
                            blocked = true;
                            r.b |= 2;
                        }
                        if (blocked) {
                            r.mask |= 1ull << q;
                            need = true;
                            simple = false;
                        } else if (st == C_ABSENT || st == C_SOLID) {
                            simple = false;
                            if (t == C_FLUID) errs[tid] = "fluid cell with a missing neighbour (a region touches a face?)";
                        }
                    }
                }
                if (t == C_CGHOST) {
                    need = true;
                    for (int q = 0; q < Q; ++q) {
                        if (q == rest) continue;
                        int64_t s[3] = {c[0] - g.lat.xi[q][0], c[1] - g.lat.xi[q][1], c[2] - g.lat.xi[q][2]};
                        int64_t sc;
                        uint8_t st = locate(i, s, sc);
                        if (!(st == C_FLUID || st == C_BC)) r.mask |= 1ull << q;
                    }
                    int64_t ch[3] = {2 * c[0], 2 * c[1], 2 * c[2]};
                    int64_t cc;
                    uint8_t ct = locate(i - 1, ch, cc);
                    if (ct != C_FGHOST) errs[tid] = "coarse ghost whose children are not fine ghosts";
                    r.a = (int32_t)cc;
                    // concave corner of the finer region: some child's two-step streaming history
                    // of an unknown population leaves the finer level (b bit 0; the kernels then
                    // test each child and let the ghost's own streamed population stand in)
                    const int nk = g.D == 3 ? 8 : 4;
                    for (int q = 0; q < Q && !(r.b & 1); ++q) {
                        if (!(r.mask >> q & 1)) continue;
                        for (int k = 0; k < nk; ++k) {
                            int64_t x[3] = {ch[0] + (k & 1), ch[1] + ((k >> 1) & 1), ch[2] + ((k >> 2) & 1)};
                            int64_t s1[3], s2[3], i1, i2;
                            for (int d = 0; d < 3; ++d) {
                                s1[d] = x[d] - g.lat.xi[q][d];
                                s2[d] = x[d] - 2 * g.lat.xi[q][d];
                            }
                            const uint8_t t1 = locate(i - 1, s1, i1);
                            if (t1 == C_ABSENT || (t1 == C_FGHOST && locate(i - 1, s2, i2) == C_ABSENT)) {
                                r.b |= 1;
                                int64_t sc[3] = {c[0] - g.lat.xi[q][0], c[1] - g.lat.xi[q][1], c[2] - g.lat.xi[q][2]};
                                int64_t scc;
                                if (locate(i, sc, scc) == C_ABSENT)
                                    errs[tid] = "a coarse ghost stands in for a fine history but has no coarse source";
                                break;
                            }
                        }
                    }
                }
                if (t == C_FGHOST || t == C_BC) {
                    int rz = g.D == 3 ? g.R : 0;
                    for (int dz = -rz; dz <= rz; ++dz)
                        for (int dy = -g.R; dy <= g.R; ++dy)
                            for (int dx = -g.R; dx <= g.R; ++dx) {
                                int64_t p[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
                                int64_t pc;
                                uint8_t pt = locate(i, p, pc);
                                if (t == C_FGHOST && pt == C_CGHOST) errs[tid] = "ghost layers closer than the lattice reach";
                                if (pt == C_SOLID) errs[tid] = "solid closer than the lattice reach to a ghost or boundary layer";
                            }
                }
                if (t == C_BC) {
                    need = true;
                    int f = g.bc_face(i, c);
                    int64_t p[3] = {c[0], c[1], c[2]};
                    for (int d = 0; d < g.D; ++d)
                        if (!g.periodic[d]) p[d] = std::min(std::max(p[d], (int64_t)g.R), lv.shape[d] - 1 - g.R);
                    int64_t pc;
                    uint8_t pt = locate(i, p, pc);
                    if (pt == C_ABSENT || pt == C_BC || pt == C_SOLID) errs[tid] = "boundary cell without an interior partner";
                    r.a = (int32_t)pc;
                    r.b = in.faces[f].kind | (f << 4);
                    r.mask = 0;
                }
                if (need) {
                    trec[tid].push_back({cell, r});
                    if (t == C_BC && in.faces[r.b >> 4].kind == BCK_NEUMANN && r.a / BS == b) neumann = true;
                    else stream = false;
                }
            }
            lv.bflag[b] = simple ? 1 : (stream ? (neumann ? 3 : 2) : 0);
        }
        for (auto& e : errs)
            if (!e.empty()) return e + " (level " + std::to_string(i) + ")";
        for (auto& v : trec)
            for (auto& pr : v) {
                lv.rec_id[pr.first] = (int32_t)lv.recs.size();
                lv.recs.push_back(pr.second);
            }
        for (int64_t k = 0; k < lv.nb * BS; ++k) lv.count[lv.type[k]]++;
        out.n_eq += double(lv.count[C_FLUID] + lv.count[C_CGHOST] + lv.count[C_FGHOST] + lv.count[C_BC]) /
                    double(int64_t(1) << i);
    }
    return std::string();
}

void grade_level_map(int dim, const int64_t* extent, int n_levels, int width, const bool* periodic, uint8_t* map) {
    int64_t e[3] = {1, 1, 1};
    for (int d = 0; d < dim; ++d) e[d] = extent[d];
    for (int i = 0; i + 1 < n_levels; ++i) {
        const int64_t f = int64_t(1) << (i + 1);          // finest cells per level-(i+1) cell
        int64_t s[3] = {1, 1, 1};
        for (int d = 0; d < dim; ++d) s[d] = e[d] / f;
        // footprint of region i at level-(i+1) resolution
        std::vector<uint8_t> foot(s[0] * s[1] * s[2], 0);
        for (int64_t z = 0; z < e[2]; ++z)
            for (int64_t y = 0; y < e[1]; ++y)
                for (int64_t x = 0; x < e[0]; ++x)
                    if (map[(z * e[1] + y) * e[0] + x] <= i)
                        foot[((dim > 2 ? z / f : 0) * s[1] + y / f) * s[0] + x / f] = 1;
        // Chebyshev dilation by `width`, one axis at a time
        for (int d = 0; d < dim; ++d) {
            std::vector<uint8_t> nxt(foot.size(), 0);
            for (int64_t z = 0; z < s[2]; ++z)
                for (int64_t y = 0; y < s[1]; ++y)
                    for (int64_t x = 0; x < s[0]; ++x) {
                        if (!foot[(z * s[1] + y) * s[0] + x]) continue;
                        int64_t c[3] = {x, y, z};
                        for (int64_t o = -width; o <= width; ++o) {
                            int64_t t[3] = {c[0], c[1], c[2]};
                            t[d] += o;
                            if (t[d] < 0 || t[d] >= s[d]) {
                                if (!periodic[d]) continue;
                                t[d] = ((t[d] % s[d]) + s[d]) % s[d];
                            }
                            nxt[(t[2] * s[1] + t[1]) * s[0] + t[0]] = 1;
                        }
                    }
            foot.swap(nxt);
        }
        for (int64_t z = 0; z < e[2]; ++z)
            for (int64_t y = 0; y < e[1]; ++y)
                for (int64_t x = 0; x < e[0]; ++x) {
                    uint8_t& v = map[(z * e[1] + y) * e[0] + x];
                    if (foot[((dim > 2 ? z / f : 0) * s[1] + y / f) * s[0] + x / f] && v > i + 1) v = (uint8_t)(i + 1);
                }
    }
}

}  // namespace lbm
