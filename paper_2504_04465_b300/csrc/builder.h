// Host grid builder of the CUDA path: level-sorted, Morton-ordered blocks of cells.
//
// Sources (arXiv 2504.04465): Sec. 3.2 (Rohde ghost layers, `reach` coarse layers overlapping
// 2*reach fine layers), Sec. 4.3 (tree, Z-order), Sec. 4.4 (level-grouped SoA storage and a
// precomputed neighbour list), Appendix A.3 (boundary layers).  The tree's single-cell leaves
// are grouped into fixed-size blocks per level so that neighbour links are stored per block
// (3^D entries) instead of per cell (Q-1 entries).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "lattice_tables.h"

namespace lbm {

enum BcKind { BCK_PERIODIC = 0, BCK_DIR = 1, BCK_DIR_RHO = 2, BCK_NEUMANN = 3, BCK_WALL = 4 };

// Per-cell record of the non-simple cells.
//   FLUID : mask = bounce-back directions (link blocked by a solid)
//   CGHOST: mask = populations supplied by coalescence; a = cell index of the child at 2c
//           in the finer level (the 2^D children are a, a+1, a+bx, a+bx+1, ... in its block)
//   BC    : a = partner cell index (same level); b = kind | face << 4
struct CellRec {
    uint64_t mask;
    int32_t a;
    int32_t b;
};

struct FaceSpec {
    int kind = BCK_PERIODIC;
    double rho = 1, u[3] = {0, 0, 0}, T = 0;
};

struct ShapeSpec {
    int kind;      // 1 sphere, 2 naca
    double p[8];
};

struct BoxSpec {
    int level;
    int64_t lo[3], hi[3];
};

struct GridInput {
    int dim = 2;
    int64_t extent[3] = {1, 1, 1};
    int n_levels = 1;
    std::vector<BoxSpec> boxes;
    // alternative to boxes: the finest level wanted at every finest-level cell (x fastest, 0 =
    // finest, n_levels - 1 = coarsest); the region of level i is then every level-(i+1) cell
    // holding a finest cell that wants level i or finer
    std::vector<uint8_t> level_map;
    std::vector<ShapeSpec> solids;
    FaceSpec faces[6];
    int block[3] = {16, 16, 1};
    int lattice = 9;
};

struct BuiltLevel {
    int level = 0;
    int64_t shape[3] = {1, 1, 1};     // cells per axis at this level
    int64_t bgrid[3] = {1, 1, 1};     // blocks per axis
    int64_t nb = 0;                   // allocated blocks
    std::vector<int32_t> bxyz;        // nb x 3 block coordinates (Morton order)
    std::vector<int32_t> nbr;         // nb x 27 neighbour blocks (offset (dx,dy,dz) -> (dx+1)+3(dy+1)+9(dz+1)), -1 if none
    std::vector<uint8_t> type;        // nb x BS
    std::vector<uint8_t> bflag;       // nb: 1 = simple (all cells fluid, every source a live non-solid cell),
                                      // 2 = streaming block (record-free fluid cells, fine ghosts, absent slots),
                                      // 0 = general
    std::vector<int32_t> rec_id;      // nb x BS: index into recs or -1
    std::vector<CellRec> recs;
    std::vector<int32_t> bindex;      // dense block grid -> block index or -1
    int64_t count[6] = {0, 0, 0, 0, 0, 0};   // cells per type
};

struct BuiltGrid {
    int dim = 2, n_levels = 1, BS = 256;
    int block[3] = {16, 16, 1};
    bool periodic[3] = {true, true, true};
    LatticeDesc lat{};
    std::vector<BuiltLevel> levels;
    double n_eq = 0;
};

// Returns an empty string on success, else a message (the grid is then unusable).
std::string build_grid(const GridInput& in, BuiltGrid& out);

// Grade a level map in place (finest resolution, x fastest): for i = 0 .. n_levels - 2, every
// level-(i+1) cell within `width` level-(i+1) cells (Chebyshev, wrapping across periodic axes) of
// a level-(i+1) cell holding a finest cell that wants level i or finer gets level i + 1 or finer,
// so that the ghost layers of consecutive interfaces keep apart (width = 3 reach + 1).
void grade_level_map(int dim, const int64_t* extent, int n_levels, int width, const bool* periodic, uint8_t* map);

}  // namespace lbm
