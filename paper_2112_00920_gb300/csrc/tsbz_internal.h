// Internal structures shared by the host runtime and the CUDA kernels.
//
// Data layout in device memory (one context):
//   psi, tA, tB : complex T, [unit][band][n3][n2][n1]; a unit is one k-point
//                 of one sub-simulation with all its bands (psi_off per unit)
//   P           : complex T, [unit][band][n_proj]          projections <beta~_j|t_b>
//   Pa          : complex T, [unit][band][n_proj][4]        <beta~_j|u>, <d_a beta~_j|u>
//   rho_part    : double,    [unit][band group][n_pts]      sum_b occ |u_b(r)|^2
//   jk_part     : double,    [unit][tile][band group][3]    sum occ Re(u* (-i grad) u)
//   nrm_part    : double,    [unit][tile][band]             sum_r |u_b(r)|^2 per tile
//   per sub-simulation: rho, v_hxc, v_eff (T), J history, J(0-), norms, step.
#pragma once
#include <cstdint>
#include <cstddef>
#include <vector_types.h>

#define TSBZ_MAX_ND 6
#define TSBZ_MAX_VARIANTS 4  // kernel variants a cell can be tuned over
#define TSBZ_PT 128        // points per CTA in the point-parallel kernels
#define TSBZ_BG 32         // max bands per band group in the point-parallel kernels
#define TSBZ_FIN_MAX_TILES 128   // most CTAs per sub-simulation of the finalize
#ifndef TSBZ_FIN_TILES
#define TSBZ_FIN_TILES 16        // CTAs per sub-simulation of the finalize (small units)
#endif

struct CellDev {
  int n1, n2, n3, npts, nmax;
  int n_atoms, n_proj, n_bands;
  int nd;
  int n_tiles;       // ceil(npts / TSBZ_PT)
  int n_bgroups;     // ceil(n_bands / TSBZ_BG)
  int use_proj;
  double dv, omega, occ;
  double lapw[3][TSBZ_MAX_ND + 1];   // c_m / h_ax^2 (m = 0..nd)
  double gradw[3][TSBZ_MAX_ND + 1];  // d_m / h_ax   (m = 1..nd)
  float hlapf[3][TSBZ_MAX_ND + 1];   // -1/2 c_m / h_ax^2 in float
  float gradwf[3][TSBZ_MAX_ND + 1];  // d_m / h_ax in float
  float2 hlap2[3][TSBZ_MAX_ND + 1];  // (w, w) pairs of hlapf for packed FP32x2 arithmetic
  float2 gradw2[3][TSBZ_MAX_ND + 1]; // (w, w) pairs of gradwf
  double gsq_scale[3];               // (2 pi / a_ax)
  const double* g1;     // [n_atoms][3][nmax] Gaussian factor exp(-d^2/(2 rc^2)), 0 outside the box
  const double* d1;     // [n_atoms][3][nmax] minimum-image displacement, 0 outside the box
  const double* pnorm;  // [n_atoms][4]        N_s, N_px, N_py, N_pz
  const double* ekb;    // [n_proj]
  const double* wkb;    // [n_proj]            pnorm_j * E_j
  const double* vloc;   // [npts]
  // the same tables in float for the single-precision kernels
  const float* g1f;
  const float* d1f;
  const float* pnormf;
  const float* wkbf;
  const float* ekbf;   // E_j
  // atoms whose z factor tables are identical (same z position, hence the same
  // Gaussian, displacement and phase rows for every q) form one z group; the
  // z contractions of the 16^3 fused stage run once per group (cells of at
  // most 8 atoms; n_zg = 0 otherwise)
  // projector boxes: per atom and axis the periodic index range [start, start + len)
  // outside which the Gaussian factor is zero ([n_atoms][3][2] ints), and whether
  // every box is at most 16 x 16 points in x and y (the box-factorised projection)
  const int* pbox;
  int pbox_ok;
  int n_zg;
  int zg_of[8];       // group of atom a
  int zg_rep[8];      // first atom of group g
  int zg_off[9];      // members of group g: zg_mem[zg_off[g] .. zg_off[g + 1])
  int zg_mem[8];
  // the same grouping for cells of up to 64 atoms in at most 8 groups (the slab
  // stage of 32-point rows; zs_n = 0 when the cell has more groups or atoms)
  int zs_n;
  int zs_off[9];      // members of group g: zs_mem[zs_off[g] .. zs_off[g + 1])
  int zs_mem[64];
};

// Whether the finalize spreads one unit over a whole CTA (units with many
// bands x projectors) rather than over one warp.
__host__ __device__ inline bool fin_wide(const CellDev& c) {
  return (long long)c.n_bands * (c.n_proj + c.n_tiles) > 4096;
}

struct UnitDev {
  long long psi_off;   // complex elements
  long long p_off;     // complex elements (P)
  long long pa_off;    // complex elements (Pa)
  long long rho_off;   // doubles
  long long jk_off;    // doubles
  long long nrm_off;   // doubles
  int sub;             // sub-simulation index
  int kloc;            // k index within the sub-simulation
};

struct SubDev {
  int cell;
  int n_k;
  int unit0;
  int max_steps;
  int n_field;         // number of field samples available (2 n + 1)
  int hxc_frozen;
  int xc, hartree;
  double dt;
  const double* A;     // [n_field][3]
  double* J;           // [max_steps + 1][3]
  double* J0m;         // [3]
  double* rho;         // [npts]
  double* vhxc;        // [npts]
  void* veff;          // [npts] in T
  double* norms;       // [n_k][n_bands]
  int* step;           // steps done
  int* status;         // non-zero: non-finite current seen
  int* active;         // 1 while the sub-simulation advances in the current step
  void* veff_save;     // [npts] in T: the other v_eff of an ETRS step (null otherwise)
  double* jtile;       // [TSBZ_FIN_MAX_TILES][3] per-tile partial sums of the current (finalize)
  int* jcount;         // tiles of the finalize done (reset by the last one)
};

// Finalize modes.
#define TSBZ_FIN_J0MINUS 0   // write J(0-)
#define TSBZ_FIN_J0PLUS 1    // write J[0] (t = 0+), only at step 0
#define TSBZ_FIN_STEP 2      // write J[step + 1] and advance the step
#define TSBZ_FIN_RHO 3       // density and norms only (ETRS predictor): no current, step unchanged
// Field modes (which q the observation tables use).
#define TSBZ_FIELD_STEP 0    // q_half = k + A(t_n + dt/2), q_obs = k + A(t_{n+1})
#define TSBZ_FIELD_J0PLUS 1  // q_obs = k + A(0+)
#define TSBZ_FIELD_J0MINUS 2 // q_obs = k
#define TSBZ_FIELD_STEP_KEEP 3  // as STEP, phase tables kept: the field is constant and they are current
#define TSBZ_FIELD_AT_NOW 4     // as STEP with the h tables at q = k + A(t_n)      (ETRS first half step)
#define TSBZ_FIELD_AT_NEXT 5    // as STEP with the h tables at q = k + A(t_{n+1})  (ETRS second half step)

struct LaunchSet {
  // Everything one kernel family needs for the units of one cell.
  CellDev cell;
  const UnitDev* units;   // global unit table
  const int* unit_ids;    // units of this cell
  int n_units;
  const SubDev* subs;
  const double* kcart;    // [unit][3]
  double* q_half;         // [unit][3]
  double* q_obs;          // [unit][3]
  void* ph_half;          // [unit][n_atoms*3*nmax] complex T
  void* ph_obs;
  void* ph_next;          // q = k + A(t_{n+1} + dt/2): tables of the next step (null if unused)
  long long ph_stride;    // complex elements per unit
  void* qt_half;          // [unit][4] in T: q_x, q_y, q_z, |q|^2 / 2 at t_n + dt/2
  int variant;            // kernel variant of this cell (0 = default; chosen by the autotuner)
  double dt_scale;        // the stage kernels advance by dt * dt_scale (1, or 1/2 in the ETRS half steps)
  const double* filt;     // [unit][3] filter coefficients of the ground-state solver (stage m = 0), or null
};

#ifdef __CUDACC__
// A unit takes part in a time step only while its sub-simulation has steps
// left in its budget; the field kernel writes the flag at the start of the step.
__device__ __forceinline__ bool unit_active(const LaunchSet& L, int u) {
  return *L.subs[L.units[u].sub].active != 0;
}
#endif

// Launchers (templated on the real type in tsbz_kernels.cuh, instantiated per precision).
template <typename T> void launch_field(const LaunchSet& L, int mode, void* stream);
template <typename T>
void launch_bra(const LaunchSet& L, const void* src, void* P, int with_d, int use_obs, void* stream);
template <typename T>
void launch_stage(const LaunchSet& L, const void* tin, void* tout, void* psi, const void* P, int m, void* stream);
template <typename T>
void launch_observe(const LaunchSet& L, const void* psi, double* rho_part, double* jk_part, double* nrm_part,
                    void* stream);
template <typename T>
void launch_finalize_t(const SubDev* subs, int n_subs, const UnitDev* units, const CellDev* cells_dev,
                       const double* q_obs, const void* Pa, const double* rho_part, const double* jk_part,
                       const double* nrm_part, const int* mask, int mode, int n_tiles, void* stream);
template <typename T>
int launch_hxc_t(const SubDev* subs_dev, const int* sub_ids_dev, int n_subs, const CellDev& c, double2* wa,
                 double2* wb, double2* const tw[3], void* stream);
template <typename T> void launch_convert_in_t(const double2* src, void* dst, long long n, void* stream);
template <typename T> void launch_convert_out_t(const void* src, double2* dst, long long n, void* stream);
template <typename T> void launch_veff_frozen_t(const SubDev* subs_dev, int s, const CellDev& c, void* stream);
template <typename T> void launch_veff_keep_t(const SubDev* subs, const CellDev* cells, int n_subs, int swap,
                                              void* stream);
// tensor-core mode (float orbitals)
void launch_bra_tc(const LaunchSet& L, const void* psi, void* out, int with_d, void* stream);
void launch_ket_tc(const LaunchSet& L, const void* P, void* V, void* stream);
bool launch_observe_zf(const LaunchSet& L, const void* psi, double* rho_part, double* jk_part, double* nrm_part,
                       void* stream);
void launch_stage_v(const LaunchSet& L, const void* tin, void* tout, void* psi, const void* V, int m, void* stream);
// single-precision fused stage and projections (cells with at most 8 atoms, depth 8 or 16, n1 n2 <= 256)
// Ground-state solver (tsbz_scf.cu).
int scf_max_bands();
void launch_scf_gram(const LaunchSet& L, const void* Y, const void* HY, void* S, void* H, void* stream);
// HY null: S only.  S, H, C, W1, W2: n_units n_b^2 complex each;
// C = L^{-H} with S + shift_coef tr(S) I = L L^H; with want_lam, H is
// replaced by L^{-1} H L^{-H} and lam receives its largest eigenvalue
void launch_scf_ortho(int n_units, int nb, double shift_coef, int want_lam, const void* S, void* H, void* C,
                      void* W1, void* W2, double* lam, int* bad, void* stream);
// Yout = Y C per unit (out of place)
void launch_scf_rotate(const LaunchSet& L, const void* Y, const void* C, void* Yout, void* stream);

// Slab z-march stage for float orbitals on grids with 32-point rows (tsbz_slab.cu):
// variant 0 of such cells; false (nothing launched) otherwise.
bool slab_supported(const CellDev& c);
bool launch_stage_slab(const LaunchSet& L, const void* tin, void* tout, void* psi, const void* P, int m,
                       void* stream);
// Observation (density, local current, band norms) of float orbitals on the same
// cells, every variant; false when the cell does not qualify.
bool launch_observe_slab(const LaunchSet& L, const void* psi, double* rho_part, double* jk_part, double* nrm_part,
                         void* stream);
// Projections of float orbitals on the same cells (variant 0): P (with_d = 0) or
// the current's Pa (with_d = 1), on the q_half (use_obs = 0) or q_obs tables;
// pnext, if given with with_d, also receives Pa's first-weight entries as P.
bool launch_bra_slab(const LaunchSet& L, const void* src, void* out, int with_d, int use_obs, void* stream,
                     void* pnext = nullptr);

bool sep_supported(const CellDev& c);
int sep_variants(const CellDev& c);   // kernel variants of the single-precision path on this cell
// The whole time step of every unit in one launch (16^3 cells with z groups,
// variant 0); false when the cell takes the per-stage kernels.
bool launch_step_fused(const LaunchSet& L, void* psi, void* P, void* Pa, int same_next, void* stream);
void launch_bra_sep(const LaunchSet& L, const void* src, void* out, int with_d, int use_obs, void* stream);
// stage 4 on the bulk-staged path also writes P (next step) and Pa; returns whether it did
// same_next: the field is constant, so at m = 4 the next step's projections come from the current's sums
bool launch_stage_sep(const LaunchSet& L, const void* tin, void* tout, void* psi, void* P, void* Pa, int m,
                      int same_next, void* stream);
bool launch_observe_fused(const LaunchSet& L, const void* psi, double* rho_part, double* jk_part, double* nrm_part,
                          void* stream);
