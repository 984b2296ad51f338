// Internal declarations shared by the host API and the kernel translation units.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "hydro.h"

namespace hydro {

constexpr int kMaxJets = 16;
constexpr int kGhost = 4;  // an interface stencil reaches 4 cells to each side (WENO7)

// Device-resident diagnostics block (one per context).
struct DevDiag {
  unsigned long long vmax_bits;   // max spectral radius of the current step, as ordered double bits
  unsigned long long floor_hits;  // cumulative primitive-recovery floor hits
  int status;                     // first hydro_status raised on the device (0 = none)
  int bad_input;                  // set by the initial-state conversion for e < 0 or non-finite input
  double dep[kMaxJets];           // per-jet RK3-weighted deposited energy [GeV]
  int cell[kMaxJets][3];          // cell where each jet deposited at its last deposit
  int check_site;                 // bounds-checked build: site of the first failed check (0 = none)
  unsigned check_index;           // and the index or coordinate it computed
};

// Jet positions for one RK stage, computed on the host in FP64.
struct JetStage {
  int n;
  int cell[kMaxJets][3];  // cell of the jet; cell[j][0] < 0: no deposit this stage
  double ell[kMaxJets];   // path length since the jet started [fm]
  double dir[kMaxJets][3];
};

// Constants of the source term (Eqs. 2-3) for one stage.
struct SourceCoef {
  double rad;     // k_rad * C_R/C_F / hbarc^2
  double coll;    // k_coll * C_R/C_F / hbarc
  double t4coef;  // T^4 = e * t4coef, t4coef = hbarc^3 / (pi^2/30 * dof)
  double inv_vol; // 1/dx^3
  double wdt_vol; // dt * RK3 weight of the stage * dx^3 (deposit diagnostic)
};

// The source constants of a configuration (Eq. 3 in natural units converted with
// hbar c, deposited per cell volume); wdt_vol is per stage and left 0.
inline SourceCoef source_coef(const hydro_config& g) {
  SourceCoef s{};
  s.rad = g.k_rad * g.cr_over_cf / (g.hbarc * g.hbarc);
  s.coll = g.k_coll * g.cr_over_cf / g.hbarc;
  s.t4coef = g.hbarc * g.hbarc * g.hbarc / (M_PI * M_PI / 30.0 * g.dof);
  s.inv_vol = 1.0 / (g.dx * g.dx * g.dx);
  return s;
}

// The launch constants in the forms the sweep kernels use, derived on the host
// (derive_constants) so that no thread converts an FP64 argument: B300 runs FP64
// arithmetic and FP64<->FP32 conversions at 1/64 of the FP32 rate.
struct LaunchConst {
  double eps_s;     // WENO epsilon in the scaled indicator form of the order in use
  float eps_s_f;    // the same rounded to FP32
  float inv_dx_f, dt_f, a_f, b_f, e_floor_f;
  float bdt_dx_f;   // b dt / dx (mixed precision: a flux difference's share of the stage increment)
  int first;        // a == 0: the stage result is U + dt L
};

// Range of the WENO epsilon each precision can represent in its weights.  FP64
// forms products of two denominators (eps_s^6 .. (eps_s + beta)^6 each); FP32
// squares reciprocals of eps_s + beta and sums four of them, so eps_s must keep
// 35 / eps_s^2 below the FP32 maximum and 1 / (eps_s + beta)^2 above its
// smallest normal.
inline bool weno_eps_ok(int precision, double eps) {
  return precision == HYDRO_FP64 ? (eps >= 1e-20 && eps <= 1e20) : (eps >= 1e-18 && eps <= 1e18);
}

// Default limit of a bounded device-side wait (hydro_config.wait_limit_s = 0), in ns.
constexpr unsigned long long kDefaultWaitNs = 250000000ull;

// The limit of a bounded wait in ns of the GPU's global timer.
inline unsigned long long wait_limit_ns(const hydro_config& c) {
  return c.wait_limit_s > 0.0 ? (unsigned long long)(c.wait_limit_s * 1e9) : kDefaultWaitNs;
}

// Configuration checks shared by every entry point.  The scheme and physics
// fields are always checked; kCheckGrid adds the grid size (nx, ny, nz >= 1,
// nx ny nz <= 4e8 for the 32-bit element indices, ny and nz <= 65535 for the
// launch-grid y and z dimensions of the single-grid sweeps); kCheckWorkspace
// the workspace alignment (256 bytes).
enum : unsigned { kCheckGrid = 1u, kCheckWorkspace = 2u };
bool config_valid(const hydro_config* c, unsigned what);

// Shu-Osher SSP-RK3 (Sec. 1): stage k evaluates L at t_n + c_k dt on U_k and forms
// U_{k+1} = a_k U^n + b_k (U_k + dt L(U_k)); w_k is the weight of L(U_k) in the
// step (the RK3-weighted deposit diagnostics).
constexpr double kRK3C[3] = {0.0, 1.0, 0.5};
constexpr double kRK3W[3] = {1.0 / 6.0, 1.0 / 6.0, 4.0 / 6.0};
constexpr double kRK3A[3] = {0.0, 0.75, 1.0 / 3.0};
constexpr double kRK3B[3] = {1.0, 0.25, 2.0 / 3.0};

// One jet at stage time t (host, FP64, without floating-point contraction: the
// library's host code compiles with -ffp-contract=off, so every entry point gets
// the same bits): path length l = t - t_start, position x = x0 + n l and cell
// floor(x/dx + N/2) per axis.  Writes the cell, or -1 on every axis when the jet
// has not started (l < 0) or lies outside the grid, and l; returns whether it
// deposits.
inline bool jet_cell_at(const double x0[3], const double n[3], double t_start, double t, double dx, const int N[3],
                        int cell[3], double* ell) {
  const double l = t - t_start;
  *ell = l;
  bool inside = (l >= 0.0);
  for (int a = 0; a < 3; ++a) {
    const double x = x0[a] + n[a] * l;
    const double fl = std::floor(x / dx + 0.5 * (double)N[a]);
    if (!(fl >= 0.0 && fl < (double)N[a])) inside = false;
    cell[a] = (fl >= 0.0 && fl < (double)N[a]) ? (int)fl : -1;
  }
  if (!inside) cell[0] = cell[1] = cell[2] = -1;
  return inside;
}

// An NVTX range over a scope: names the library's calls and RK3 stages on a
// profiler's timeline (ncu --nvtx, Nsight Systems); without an attached tool the
// push and pop return at once.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Everything a sweep tile needs except the jet list.
struct GridArgs {
  const void* U;    // state the right-hand side is evaluated on
  const void* U0;   // state at the start of the step (stage combination)
  void* Uout;       // combined stage result (z sweep only)
  void* rhs;        // right-hand-side accumulator
  const float* S;   // mixed precision: FP32 shadow of U ([6][n], mixed_shadow), or NULL.  With
                    // it the accumulator holds delta_k = U_k - U0 between stages and the z
                    // sweep writes U (into Uout = U0) only at the last stage (Uout != NULL)
  float* Sout;      // mixed precision: shadow of the stage result, written by the z sweep (with S)
  void* P;          // FP64: primitives the x sweep recovers, cached for the y and z sweeps of the
                    // same stage: [5][n], v_y, rho_y, p, v_z, rho_z (NULL: every sweep recovers its
                    // staged cells itself, as FP32 and mixed precision do)
  DevDiag* diag;
  int nx, ny, nz;
  int periodic;
  double inv_dx;
  double dt;
  double a, b;      // Uout = a U0 + b (U + dt L)
  double e_floor;
  double eps;       // WENO epsilon
  int reduce_speed; // 1: fold spectral radii into diag->vmax_bits
  int count_floors; // 1: count floor hits (x sweep of each stage)
  unsigned long long wait_ns;  // limit of each bounded wait on a TMA copy (0: kDefaultWaitNs)
  int withhold;     // fault injection: arm the copy barriers but issue no TMA copy
  int check_tighten;  // bounds-checked build: halve every checked bound (test hook)
  SourceCoef src;
  LaunchConst k;    // filled by the launchers from the fields above
};

// The fields of a sweep launch that follow from the configuration alone (grid,
// boundary, step, floor, epsilon, source constants, wait limit, test hooks); the
// buffers, the diagnostics block and the per-stage fields are the caller's.
inline void grid_args_from_config(const hydro_config& g, GridArgs& a) {
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.periodic = g.boundary == HYDRO_PERIODIC;
  a.inv_dx = 1.0 / g.dx;
  a.dt = g.dt;
  a.e_floor = g.e_floor;
  a.eps = g.weno_eps;
  a.src = source_coef(g);
  a.wait_ns = wait_limit_ns(g);
  a.withhold = g.test_withhold_copies;
  a.check_tighten = g.test_check_tighten;
}

// Arguments of a single-grid sweep launch.
struct SweepArgs : GridArgs {
  JetStage jets;
};

// One grid of a batched ensemble: its size and where its fields start.
struct BatchEvent {
  int nx, ny, nz;
  int pad;
  size_t off;       // element offset of the grid's 5 fields in every state array
};

struct SweepMaps;

// Arguments of a batched sweep launch: one launch covers every tile of every
// grid; a tile is two int4, (event, a0, l0, fixed) and (nx, ny, nz, first cell of
// the grid in the concatenated arrays).
struct BatchArgs {
  const BatchEvent* events;
  const int4* tiles;   // 2 ntiles entries
  int ntiles;
  int periodic;
  const void* U;    // base of the concatenated state arrays
  const void* U0;
  void* Uout;       // mixed precision: NULL except at the last stage (see GridArgs::S)
  void* rhs;
  const float* S;   // mixed precision: bases of the concatenated shadows (event e's [6][n_e] block
  float* Sout;      // starts at 6/5 of its state offset); NULL otherwise
  void* P;          // cached primitives, laid out like the accumulator (see GridArgs::P), or NULL
  DevDiag* diags;   // one per event
  const JetStage* jets;   // one per event, for this stage
  double inv_dx, dt, a, b, e_floor, eps;
  int reduce_speed, count_floors;
  unsigned long long wait_ns;   // limit of each bounded wait on a TMA copy (0: kDefaultWaitNs)
  int withhold;     // fault injection: arm the copy barriers but issue no TMA copy
  int check_tighten;  // bounds-checked build: halve every checked bound (test hook)
  SourceCoef src;
  LaunchConst k;    // filled by launch_batch_sweep
  const SweepMaps* maps;   // [nev] tensor maps of this launch's stage and axis, or NULL (plain loads)
};

// Tile shapes the batched sweeps can use (index = autotuner choice):
// x sweep (SEG along x, LANES rows), y and z sweeps (SEG along the axis, LANES x-lanes).
constexpr int kBatchVariants = 3;
constexpr int kTileSegX[kBatchVariants] = {64, 32, 128};
constexpr int kTileLanesX[kBatchVariants] = {4, 8, 2};
constexpr int kTileSegYZ[kBatchVariants] = {32, 16, 64};
constexpr int kTileLanesYZ[kBatchVariants] = {8, 16, 4};

cudaError_t launch_batch_sweep(int precision, int dir, int variant, const BatchArgs& a, int grid, cudaStream_t s);
// Blocks per SM the batched sweep kernel (with or without tensor maps) reaches (0 on error).
int batch_sweep_blocks_per_sm(int precision, int dir, int variant, bool tma);

// Tensor maps of a batched ensemble, maps[(stage * 3 + axis) * nev + event], for the tile
// shapes variant[axis]; bufs[st] are the concatenated state arrays, rhs the accumulator,
// off[e] the element offset of event e's fields, shadows[st] (mixed precision) the
// concatenated shadows.  False when a grid misses the TMA layout rules (row pitch and
// field offset multiples of 16 bytes); callers then launch the plain-load kernels.
bool encode_batch_tmaps(int precision, void* const bufs[3], void* rhs, int nev, const int32_t* dims,
                        const size_t* off, const int variant[3], SweepMaps* maps, void* const shadows[3] = nullptr);
// Zeroes the per-step maximum signal speed of n diagnostics blocks.
cudaError_t launch_reset_vmax(DevDiag* diags, int n, cudaStream_t s);

// Tensor maps of one sweep launch: `stage` boxes the staged cells of a tile in
// the state the right-hand side is evaluated on (FP64 and FP32) or in its FP32
// shadow (mixed); `rhs` and `u0` box the tile's updated cells in the accumulator
// and the step state.  FP32-flux (FP32, mixed) sweeps fetch their phase-3
// operands through them (y and z) and store their accumulator values through
// `rhs` (x, y).
struct SweepMaps {
  CUtensorMap stage, rhs, u0;
};

// Launches one directional sweep (dir 0/1/2) for the given precision
// (0 FP64, 1 FP32, 2 mixed) and WENO order (7 or 5).
// maps (may be NULL): the tensor maps of this stage and sweep axis from
// encode_sweep_tmaps; with them, tiles that need no ghost cells are staged by TMA
// and the phase-3 operands arrive by TMA.
cudaError_t launch_sweep(int precision, int order, int dir, const SweepArgs& a, cudaStream_t s,
                         const SweepMaps* maps = nullptr);

// Tensor maps for the three RK stages and the three sweep axes (maps[stage][axis]);
// bufs[st] is the state stage st evaluates its right-hand side on (bufs[0] is also
// the step state U0), rhs the accumulator.  WENO7 and WENO5.  Returns false (and leaves
// maps unusable) when the grid does not meet the TMA layout rules (row pitch a
// multiple of 16 bytes) or the driver entry point is missing; callers then use
// plain loads.
// shadows: for mixed precision (required there; NULL otherwise), the FP32 shadows
// [6][n] of the three stage states, whose staging boxes go into the maps' `stage`
// entries.
bool encode_sweep_tmaps(int precision, int order, void* const bufs[3], void* rhs, int nx, int ny, int nz,
                        SweepMaps maps[3][3], void* const shadows[3] = nullptr);

// Mixed precision: the FP32 shadow [6][n] of an FP64 state [5][n] (the sweeps'
// staging input; see mixed_shadow).
cudaError_t launch_shadow(const double* U, float* S, size_t n, double e_floor, cudaStream_t s);

// Initial state: staging (5N FP64, prim or cons) -> conserved state in storage precision.
cudaError_t launch_init(int precision, int kind, const double* staging, void* U, size_t n, DevDiag* diag,
                        cudaStream_t s);

// Read-back: state in storage precision -> 5N FP64 (conserved, or primitive with u^i).
cudaError_t launch_readback(int precision, int kind, const void* U, double* staging, size_t n, double e_floor,
                            cudaStream_t s);

}  // namespace hydro
