// hydro_step_noalloc: RK3 steps on a caller-owned device state without any
// device allocation.
//
// Who needs this: callers that cannot call cudaMalloc -- code running inside
// a memory pool or arena it does not own, a plugin whose host forbids device
// allocation after start-up, or a real-time loop where an allocation's
// latency (or its failure) is not acceptable.  hydro_create needs a workspace
// (three state copies, a right-hand-side accumulator and a primitive cache);
// this entry point instead keeps the two intermediate RK3 stages, the
// accumulator, the cache and the diagnostics block in one fixed array compiled
// into the library.
//
// Cost of that choice: every GPU that loads the library holds the array
// (kScratchBytes, about 10.5 MB) until the process exits, the grid is limited
// to kNoAllocMaxCells cells, and all calls share the array, so calls whose
// work overlaps on the GPU (different streams or threads sharing the device)
// race on it and must be serialised by the caller.
//
// The array's name is only a host-side stand-in for the symbol: the device
// address is looked up with cudaGetSymbolAddress once per device (on the
// first call made with that device current) and passed to the kernels.
#include <cmath>
#include <cstring>
#include <mutex>

#include "hydro.h"
#include "hydro_internal.h"

namespace {

using hydro::DevDiag;
using hydro::SweepArgs;

constexpr size_t kNoAllocMaxCells = HYDRO_NOALLOC_MAX_CELLS;
constexpr size_t kAlign = 256;
constexpr size_t kStateBytesMax = ((5 * kNoAllocMaxCells * sizeof(double) + kAlign - 1) / kAlign) * kAlign;
constexpr size_t kDiagBytes = ((sizeof(DevDiag) + kAlign - 1) / kAlign) * kAlign;
// two stage states, the accumulator and (FP64) the x sweep's primitive cache at
// FP64 width, then the diagnostics block; mixed precision instead keeps three
// FP32 shadows of 6 fields and an FP32 accumulator (6 + 6 + 6 + 5 floats per
// cell), which fit in the same space
constexpr size_t kScratchBytes = 4 * kStateBytesMax + kDiagBytes;
constexpr size_t kShadowBytesMax = ((6 * kNoAllocMaxCells * sizeof(float) + kAlign - 1) / kAlign) * kAlign;
static_assert(3 * kShadowBytesMax + kStateBytesMax <= 4 * kStateBytesMax, "mixed layout fits the scratch array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
hydro_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HYDRO_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return HYDRO_ECUDA;
    }
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return HYDRO_OK;
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// The checks of hydro_create (grid size and launch limits included); the
// workspace field is ignored here.
bool config_ok(const hydro_config* c) { return hydro::config_valid(c, hydro::kCheckGrid); }

}  // namespace

extern "C" hydro_status hydro_step_noalloc(const hydro_config* cfg, void* d_state, int64_t step0, int32_t nsteps,
                                           const double* jets, int32_t njet, hydro_diag* diag_out) {
  if (!config_ok(cfg) || !d_state || nsteps < 0 || step0 < 0) return HYDRO_EINVAL;
  if (njet < 0 || njet > HYDRO_MAX_JETS || (njet > 0 && !jets)) return HYDRO_EINVAL;
  const size_t n = (size_t)cfg->nx * (size_t)cfg->ny * (size_t)cfg->nz;
  if (n > kNoAllocMaxCells) return HYDRO_ENOMEM;   // the fixed scratch array is too small for this grid
  const size_t store = cfg->precision == HYDRO_FP32 ? sizeof(float) : sizeof(double);
  if ((uintptr_t)d_state % store != 0) return HYDRO_EINVAL;

  // jets: x0[3], dir[3], t_start per jet; the direction is normalised as in hydro_add_jet
  double jx0[HYDRO_MAX_JETS][3], jn[HYDRO_MAX_JETS][3], jt[HYDRO_MAX_JETS];
  for (int j = 0; j < njet; ++j) {
    const double* r = jets + 7 * j;
    for (int a = 0; a < 7; ++a)
      if (!std::isfinite(r[a])) return HYDRO_EINVAL;
    const double len = std::sqrt(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
    if (!(len > 0.0)) return HYDRO_EINVAL;
    for (int a = 0; a < 3; ++a) {
      jx0[j][a] = r[a];
      jn[j][a] = r[3 + a] / len;
    }
    jt[j] = r[6];
  }

  void* base = nullptr;
  hydro_status st = scratch_address(&base);
  if (st != HYDRO_OK) return st;
  char* b = static_cast<char*>(base);
  const bool mixed = cfg->precision == HYDRO_MIXED;
  void* U1 = b;
  void* U2 = b + align_up(5 * n * store);
  void* rhs = b + 2 * align_up(5 * n * store);
  void* prim = cfg->precision == HYDRO_FP64 ? b + 3 * align_up(5 * n * store) : nullptr;
  float* S[3] = {nullptr, nullptr, nullptr};
  if (mixed) {   // the shadows of the stage states, then the FP32 accumulator
    for (int k = 0; k < 3; ++k) S[k] = reinterpret_cast<float*>(b + k * align_up(6 * n * sizeof(float)));
    rhs = b + 3 * align_up(6 * n * sizeof(float));
  }
  DevDiag* diag = reinterpret_cast<DevDiag*>(b + 4 * kStateBytesMax);
  cudaStream_t stream = static_cast<cudaStream_t>(cfg->cuda_stream);

  // the diagnostics block keeps the previous call's contents: start from zero
  cudaError_t err = cudaMemsetAsync(diag, 0, sizeof(DevDiag), stream);
  // mixed precision stages the FP32 shadow of the caller's state
  if (err == cudaSuccess && mixed && nsteps > 0)
    err = hydro::launch_shadow(static_cast<const double*>(d_state), S[0], n, cfg->e_floor, stream);

  void* U[3] = {d_state, U1, U2};
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.U0 = d_state;
  a.rhs = rhs;
  a.P = prim;
  a.diag = diag;
  hydro::grid_args_from_config(*cfg, a);   // (plain loads: no TMA copy and no wait here)
  const double vol = cfg->dx * cfg->dx * cfg->dx;
  const int N[3] = {cfg->nx, cfg->ny, cfg->nz};
  for (int32_t s = 0; s < nsteps && err == cudaSuccess; ++s) {
    const int64_t step = step0 + s;
    err = cudaMemsetAsync(&diag->vmax_bits, 0, sizeof(unsigned long long), stream);
    for (int k = 0; k < 3 && err == cudaSuccess; ++k) {
      const double t = cfg->t0 + ((double)step + hydro::kRK3C[k]) * cfg->dt;
      a.jets.n = njet;
      for (int j = 0; j < njet; ++j) {
        hydro::jet_cell_at(jx0[j], jn[j], jt[j], t, cfg->dx, N, a.jets.cell[j], &a.jets.ell[j]);
        for (int ax = 0; ax < 3; ++ax) a.jets.dir[j][ax] = jn[j][ax];
      }
      a.src.wdt_vol = cfg->dt * hydro::kRK3W[k] * vol;
      a.U = U[k];
      a.Uout = (k == 2) ? U[0] : U[k + 1];
      if (mixed) {   // stage states as FP32 increments over U0 in the accumulator, as hydro_step
        a.U = U[0];
        a.Uout = k == 2 ? U[0] : nullptr;
        a.S = S[k];
        a.Sout = S[k == 2 ? 0 : k + 1];
      }
      a.a = hydro::kRK3A[k];
      a.b = hydro::kRK3B[k];
      a.reduce_speed = (k == 0);
      for (int dir = 0; dir < 3 && err == cudaSuccess; ++dir) {
        a.count_floors = (dir == 0);
        err = hydro::launch_sweep(cfg->precision, cfg->weno_order, dir, a, stream);
      }
    }
  }
  if (err != cudaSuccess) return HYDRO_ECUDA;
  DevDiag d;
  err = cudaMemcpyAsync(&d, diag, sizeof(d), cudaMemcpyDeviceToHost, stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
  if (err != cudaSuccess) return HYDRO_ECUDA;
  if (diag_out) {
    std::memset(diag_out, 0, sizeof(*diag_out));
    diag_out->t = cfg->t0 + (double)(step0 + nsteps) * cfg->dt;
    diag_out->steps = step0 + nsteps;
    std::memcpy(&diag_out->max_speed, &d.vmax_bits, sizeof(double));
    diag_out->floor_hits = (int64_t)d.floor_hits;
    diag_out->njet = njet;
    for (int j = 0; j < HYDRO_MAX_JETS; ++j)
      for (int ax = 0; ax < 3; ++ax) diag_out->jet_cell[j][ax] = j < njet ? d.cell[j][ax] : -1;
    for (int j = 0; j < njet; ++j) {
      diag_out->dep_E += d.dep[j];
      for (int ax = 0; ax < 3; ++ax) diag_out->dep_M[ax] += jn[j][ax] * d.dep[j];
    }
    diag_out->status = d.status;
    diag_out->check_site = d.check_site;
    diag_out->check_index = d.check_index;
  }
  if (d.status != 0) return (hydro_status)d.status;
  if (cfg->cfl_limit > 0.0 && nsteps > 0) {
    double vmax;
    std::memcpy(&vmax, &d.vmax_bits, sizeof(vmax));
    if (vmax * cfg->dt / cfg->dx > cfg->cfl_limit) return HYDRO_ECFL;
  }
  return HYDRO_OK;
}
