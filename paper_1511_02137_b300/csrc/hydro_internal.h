// Internal declarations shared by the host API and the kernel translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

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

struct SweepArgs {
  const void* U;    // state the right-hand side is evaluated on
  const void* U0;   // state at the start of the step (stage combination)
  void* Uout;       // combined stage result (z sweep only)
  void* rhs;        // right-hand-side accumulator
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
  JetStage jets;
  SourceCoef src;
};

// Launches one directional sweep (dir 0/1/2) for the given precision
// (0 FP64, 1 FP32, 2 mixed) and WENO order (7 or 5).
cudaError_t launch_sweep(int precision, int order, int dir, const SweepArgs& a, cudaStream_t s);

// Initial state: staging (5N FP64, prim or cons) -> conserved state in storage precision.
cudaError_t launch_init(int precision, int kind, const double* staging, void* U, size_t n, DevDiag* diag,
                        cudaStream_t s);

// Read-back: state in storage precision -> 5N FP64 (conserved, or primitive with u^i).
cudaError_t launch_readback(int precision, int kind, const void* U, double* staging, size_t n, double e_floor,
                            cudaStream_t s);

}  // namespace hydro
