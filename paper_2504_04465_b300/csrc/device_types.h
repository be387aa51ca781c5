// Launch descriptors shared by the host scheduler (api.cpp) and the kernels.
#pragma once
#include <cstdint>

namespace lbm {

constexpr int MAX_LEVELS = 8;
enum : int { ST_F64 = 1, ST_F32 = 2, ST_F16DEV = 3 };

struct CellRecDev {
    unsigned long long mask;
    int a;
    int b;
};

struct LevelDev {
    long long nb;            // blocks
    long long ncell;         // nb * BS: SoA stride
    const int* nbr;          // nb * 27
    const unsigned char* type;
    const unsigned char* bflag;   // 1 simple, 2 streaming, 3 streaming with Neumann boundary cells, 0 general
    const int* rec_id;
    const CellRecDev* recs;
    void* f[2];
    void* g[2];
    double* lam;             // 2 buffers x 8 x ncell (numerical equilibrium)
    double tau;
    double omega;            // 1 / tau
    float omega_f;           // 1 / tau in FP32 (no division in the kernels)
    double omega_m;          // two-relaxation-time collision: rate of the odd part
    float omega_m_f;
    const int* bxyz;         // block coordinates (3 per block), for position-dependent terms
    int shape[3];            // cells per axis of the level
    const int* blist[2];     // [0] 4 * block + s: simple (s = 0), streaming (s = 1) and streaming blocks with
                             // Neumann boundary cells (s = 3), [1] the others
                             // (block nb of f/g holds zero populations: the missing-neighbour stand-in)
    long long nlist[2];
};

struct FaceDev {
    int kind;
    double rho, u[3], T;
};

struct ModelDev {
    double cs2;              // theta of the viscosity relation
    double T0;               // reference temperature (compressible)
    double Cv;               // 1/(gamma - 1)
    double rho_ref;          // F16DEV reference density
    float rho_ref_f, inv_rho_ref_f;   // the same in FP32, and its reciprocal
    float gref_f, inv_gref_f;         // g reference rho_ref (2 Cv - D) T0 in FP32, and its reciprocal
    int sensor_on;
    double sensor_A;
    double newton_tol;
    int newton_max_iter;
    int newton_fp32;         // Newton arithmetic in FP32
    int guess;
    FaceDev faces[6];
    const float* mlp;        // Newton-guess network (bf16-rounded weights), guess == 3
    int sponge_on;           // far-field relaxation (weakly compressible models)
    double sp_c[3], sp_r0, sp_r1, sp_smax, sp_rho_inf;   // its centre, radii (finest units), sigma_max, rho_inf
    double mlp_m[8], mlp_s[8];
};

struct StepArgs {
    LevelDev lv[MAX_LEVELS];
    int n_levels;
    int n_active;
    int active[MAX_LEVELS];           // active levels, coarsest first
    long long block_off[MAX_LEVELS + 1];      // over all blocks of the active levels
    long long list_off[2][MAX_LEVELS + 1];    // over the simple / other block lists
    int rd[MAX_LEVELS];               // buffer index read by each level this iteration
    int sync_fg[MAX_LEVELS];          // 1: the level's fine ghosts receive an explosion now
    int aa;                           // AA-pattern streaming: one population buffer (single level)
    int aa_l1;                        // readout: the buffer holds layout L1 (own slot qbar = f_q)
    ModelDev m;
    int* status;                      // first error code (atomicCAS from 0)
    unsigned long long* nstat;        // newton: [0] iter sum, [1] updates, [2] nonconverged, [3..18] hist
};

}  // namespace lbm
