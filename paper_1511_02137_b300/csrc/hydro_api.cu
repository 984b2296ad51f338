// Host side of the C ABI declared in include/hydro.h: configuration checks,
// the device workspace (field store), the jet list, the SSP-RK3 stage driver
// and diagnostics.  All device work goes through the kernels in
// hydro_sweep.cu; there is no host fallback.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "hydro.h"
#include "hydro_internal.h"

using namespace hydro;

bool hydro::config_valid(const hydro_config* c, unsigned what) {
  if (!c) return false;
  if (what & kCheckGrid) {
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) return false;
    if ((double)c->nx * c->ny * c->nz > 4.0e8) return false;   // 32-bit grid indices, 5 fields
    if (c->nz > 65535 || c->ny > 65535) return false;          // grid z/y launch limits
  }
  if (c->precision < HYDRO_FP64 || c->precision > HYDRO_MIXED) return false;
  if (c->boundary != HYDRO_OUTFLOW && c->boundary != HYDRO_PERIODIC) return false;
  if (c->weno_order != 7 && c->weno_order != 5) return false;
  if (!(c->dx > 0.0) || !(c->dt > 0.0) || !std::isfinite(c->t0)) return false;
  if (!(c->hbarc > 0.0) || !(c->dof > 0.0) || !(c->e_floor > 0.0) || !weno_eps_ok(c->precision, c->weno_eps)) return false;
  if (!std::isfinite(c->k_rad) || !std::isfinite(c->k_coll) || !std::isfinite(c->cr_over_cf)) return false;
  if (!(c->wait_limit_s >= 0.0 && c->wait_limit_s <= 10.0)) return false;
  if (c->test_withhold_copies != 0 && c->test_withhold_copies != 1) return false;
#ifdef HYDRO_CHECK
  if (c->test_check_tighten != 0 && c->test_check_tighten != 1) return false;
#else
  if (c->test_check_tighten != 0) return false;   // a hook of the bounds-checked build only
#endif
  if ((what & kCheckWorkspace) && c->workspace && ((uintptr_t)c->workspace % 256) != 0) return false;
  return true;
}

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

size_t store_bytes(int precision) { return precision == HYDRO_FP32 ? 4 : 8; }
size_t flux_bytes(int precision) { return precision == HYDRO_FP64 ? 8 : 4; }

struct Layout {
  size_t u0, u1, u2, rhs, prim, diag, s[3], total;
};

// Three states and the accumulator, in FP64 the primitives the x sweep caches for
// the y and z sweeps, the diagnostics block, and for mixed precision the FP32
// shadows [6][n] of the three states that the sweeps stage.
Layout layout_for(const hydro_config& c) {
  const size_t n = (size_t)c.nx * c.ny * c.nz;
  const size_t state = align_up(5 * n * store_bytes(c.precision));
  Layout L;
  L.u0 = 0;
  L.u1 = L.u0 + state;
  L.u2 = L.u1 + state;   // u1 .. u2 end also serves as the 5n-double host-transfer staging area
  L.rhs = L.u2 + state;
  // FP64: the primitives the x sweep caches for the y and z sweeps (in FP32 and
  // mixed precision the sweeps recover their staged cells faster than they load them)
  L.prim = L.rhs + align_up(5 * n * flux_bytes(c.precision));
  L.diag = L.prim + (c.precision == HYDRO_FP64 ? align_up(5 * n * sizeof(double)) : 0);
  size_t off = L.diag + align_up(sizeof(DevDiag));
  for (int k = 0; k < 3; ++k) {
    L.s[k] = off;
    if (c.precision == HYDRO_MIXED) off += align_up(6 * n * sizeof(float));
  }
  L.total = off;
  return L;
}

bool config_ok(const hydro_config* c) { return config_valid(c, kCheckGrid | kCheckWorkspace); }

struct Prof {
  std::vector<cudaEvent_t> ev[HYDRO_KERNEL_COUNT];   // start/stop pairs, resolved at query time
  double ms[HYDRO_KERNEL_COUNT] = {0, 0, 0, 0};
  int64_t n[HYDRO_KERNEL_COUNT] = {0, 0, 0, 0};
};

}  // namespace

struct hydro_ctx {
  hydro_config cfg;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  bool owns_ws = false;
  Layout lay;
  size_t n = 0;
  bool initialized = false;
  int64_t steps = 0;
  int njet = 0;
  double jx0[kMaxJets][3];
  double jn[kMaxJets][3];
  double jt[kMaxJets];
  bool profiling = false;
  Prof prof;
  SweepMaps tmaps[3][3];     // [stage][sweep axis], valid when tma
  bool tma = false;
  void* U(size_t off) { return ws + off; }
  DevDiag* diag() { return reinterpret_cast<DevDiag*>(ws + lay.diag); }
  double* staging() { return reinterpret_cast<double*>(ws + lay.u1); }
  float* shadow(int k) { return cfg.precision == HYDRO_MIXED ? reinterpret_cast<float*>(ws + lay.s[k]) : nullptr; }
};

namespace {

hydro_status cuda_status(cudaError_t e) { return e == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA; }

void prof_clear(hydro_ctx* c) {
  for (int k = 0; k < HYDRO_KERNEL_COUNT; ++k) {
    for (cudaEvent_t e : c->prof.ev[k]) cudaEventDestroy(e);
    c->prof.ev[k].clear();
    c->prof.ms[k] = 0.0;
    c->prof.n[k] = 0;
  }
}

// Records an event before (start = true) or after a launch of kernel kind k.
void prof_mark(hydro_ctx* c, int k) {
  if (!c->profiling) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, c->stream);
  c->prof.ev[k].push_back(e);
}

hydro_status prof_resolve(hydro_ctx* c) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HYDRO_ECUDA;
  for (int k = 0; k < HYDRO_KERNEL_COUNT; ++k) {
    auto& v = c->prof.ev[k];
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, v[i], v[i + 1]) == cudaSuccess) {
        c->prof.ms[k] += ms;
        c->prof.n[k] += 1;
      }
    }
    for (cudaEvent_t e : v) cudaEventDestroy(e);
    v.clear();
  }
  return HYDRO_OK;
}

// Cell of jet j at stage time t (host, FP64, no contraction): x = x0 + n (t - t_start),
// index floor(x/dx + N/2) per axis.  Returns false when the jet has not started
// or lies outside the grid.
bool jet_cell(const hydro_ctx* c, int j, double t, int cell[3], double* ell) {
  const int N[3] = {c->cfg.nx, c->cfg.ny, c->cfg.nz};
  return jet_cell_at(c->jx0[j], c->jn[j], c->jt[j], t, c->cfg.dx, N, cell, ell);
}

}  // namespace

extern "C" {

void hydro_config_default(hydro_config* c, int32_t nx, int32_t ny, int32_t nz) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->precision = HYDRO_FP64;
  c->boundary = HYDRO_OUTFLOW;
  c->weno_order = 7;
  c->dx = 0.1;
  c->dt = 0.02;
  c->t0 = 1.0;
  c->k_rad = 4.0;
  c->k_coll = 2.5;
  c->cr_over_cf = 1.0;
  c->hbarc = 0.1973;
  c->dof = 47.5;
  c->e_floor = 3e-11;
  c->weno_eps = 1e-6;
  c->cfl_limit = 1.0;
}

hydro_status hydro_workspace_size(const hydro_config* cfg, size_t* bytes) {
  if (!config_ok(cfg) || !bytes) return HYDRO_EINVAL;
  *bytes = layout_for(*cfg).total;
  return HYDRO_OK;
}

hydro_status hydro_create(const hydro_config* cfg, hydro_ctx** out) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  if (!config_ok(cfg)) return HYDRO_EINVAL;
  hydro_ctx* c = new (std::nothrow) hydro_ctx;
  if (!c) return HYDRO_ENOMEM;
  c->cfg = *cfg;
  c->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  c->lay = layout_for(*cfg);
  c->n = (size_t)cfg->nx * cfg->ny * cfg->nz;
  if (cfg->workspace) {
    if (cfg->workspace_bytes < c->lay.total) {
      delete c;
      return HYDRO_ENOMEM;
    }
    c->ws = static_cast<char*>(cfg->workspace);
  } else {
    if (cudaMalloc(&c->ws, c->lay.total) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return HYDRO_ENOMEM;
    }
    c->owns_ws = true;
  }
  if (cudaMemsetAsync(c->diag(), 0, sizeof(DevDiag), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    hydro_destroy(c);
    return HYDRO_ECUDA;
  }
  void* bufs[3] = {c->U(c->lay.u0), c->U(c->lay.u1), c->U(c->lay.u2)};
  void* shadows[3] = {c->shadow(0), c->shadow(1), c->shadow(2)};
  c->tma = encode_sweep_tmaps(cfg->precision, cfg->weno_order, bufs, c->U(c->lay.rhs), cfg->nx, cfg->ny, cfg->nz,
                              c->tmaps, cfg->precision == HYDRO_MIXED ? shadows : nullptr);
  *out = c;
  return HYDRO_OK;
}

hydro_status hydro_set_initial(hydro_ctx* c, int32_t kind, const double* host5) {
  if (!c || !host5 || (kind != HYDRO_PRIMITIVE && kind != HYDRO_CONSERVED)) return HYDRO_EINVAL;
  const size_t n = c->n;
  DevDiag zero;
  std::memset(&zero, 0, sizeof(zero));
  cudaError_t e = cudaMemcpyAsync(c->diag(), &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->staging(), host5, 5 * n * sizeof(double), cudaMemcpyDefault, c->stream);   // host or device
  if (e != cudaSuccess) return HYDRO_ECUDA;
  prof_mark(c, HYDRO_KERNEL_OTHER);
  e = launch_init(c->cfg.precision, kind, c->staging(), c->U(c->lay.u0), n, c->diag(), c->stream);
  if (e == cudaSuccess && c->cfg.precision == HYDRO_MIXED)
    e = launch_shadow(static_cast<const double*>(c->U(c->lay.u0)), c->shadow(0), n, c->cfg.e_floor, c->stream);
  prof_mark(c, HYDRO_KERNEL_OTHER);
  if (e != cudaSuccess) return HYDRO_ECUDA;
  int bad = 0;
  e = cudaMemcpyAsync(&bad, &c->diag()->bad_input, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return HYDRO_ECUDA;
  if (bad) {
    c->initialized = false;
    return HYDRO_EINVAL;
  }
  c->initialized = true;
  c->steps = 0;
  return HYDRO_OK;
}

hydro_status hydro_add_jet(hydro_ctx* c, const double x0[3], const double dir[3], double t_start,
                           int32_t* jet_id) {
  if (!c || !x0 || !dir || !std::isfinite(t_start)) return HYDRO_EINVAL;
  if (c->njet >= kMaxJets) return HYDRO_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(x0[a]) || !std::isfinite(dir[a])) return HYDRO_EINVAL;
  const double len = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (!(len > 0.0) || !std::isfinite(len)) return HYDRO_EINVAL;
  const int j = c->njet++;
  for (int a = 0; a < 3; ++a) {
    c->jx0[j][a] = x0[a];
    c->jn[j][a] = dir[a] / len;
  }
  c->jt[j] = t_start;
  if (jet_id) *jet_id = j;
  return HYDRO_OK;
}

hydro_status hydro_step(hydro_ctx* c, int32_t nsteps) {
  if (!c || nsteps < 0) return HYDRO_EINVAL;
  if (!c->initialized) return HYDRO_ESTATE;
  NvtxRange call("hydro_step");
  static const char* const kStageName[3] = {"rk3 stage 1", "rk3 stage 2", "rk3 stage 3"};
  const hydro_config& g = c->cfg;
  void* U[3] = {c->U(c->lay.u0), c->U(c->lay.u1), c->U(c->lay.u2)};
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.U0 = U[0];
  a.rhs = c->U(c->lay.rhs);
  a.P = g.precision == HYDRO_FP64 ? c->U(c->lay.prim) : nullptr;
  a.diag = c->diag();
  grid_args_from_config(g, a);
  const double vol = g.dx * g.dx * g.dx;
  cudaError_t err = cudaSuccess;
  for (int32_t s = 0; s < nsteps && err == cudaSuccess; ++s) {
    const int64_t n = c->steps;
    err = cudaMemsetAsync(&c->diag()->vmax_bits, 0, sizeof(unsigned long long), c->stream);
    for (int st = 0; st < 3 && err == cudaSuccess; ++st) {
      NvtxRange stage(kStageName[st]);
      const double t = g.t0 + ((double)n + kRK3C[st]) * g.dt;
      a.jets.n = c->njet;
      for (int j = 0; j < c->njet; ++j) {
        jet_cell(c, j, t, a.jets.cell[j], &a.jets.ell[j]);
        for (int d = 0; d < 3; ++d) a.jets.dir[j][d] = c->jn[j][d];
      }
      a.src.wdt_vol = g.dt * kRK3W[st] * vol;
      a.U = U[st];
      a.Uout = (st == 2) ? U[0] : U[st + 1];
      a.S = c->shadow(st);                        // NULL unless mixed precision
      a.Sout = c->shadow(st == 2 ? 0 : st + 1);
      if (a.S) {
        // mixed: stage states as FP32 increments over U0 in the accumulator, the
        // FP64 state written at the last stage only
        a.U = U[0];
        a.Uout = st == 2 ? U[0] : nullptr;
      }
      a.a = kRK3A[st];
      a.b = kRK3B[st];
      a.reduce_speed = (st == 0);
      for (int dir = 0; dir < 3 && err == cudaSuccess; ++dir) {
        a.count_floors = (dir == 0);
        prof_mark(c, HYDRO_KERNEL_SWEEP_X + dir);
        err = launch_sweep(g.precision, g.weno_order, dir, a, c->stream, c->tma ? &c->tmaps[st][dir] : nullptr);
        prof_mark(c, HYDRO_KERNEL_SWEEP_X + dir);
      }
    }
    if (err == cudaSuccess) c->steps += 1;
  }
  if (err != cudaSuccess) return HYDRO_ECUDA;
  DevDiag d;
  err = cudaMemcpyAsync(&d, c->diag(), sizeof(d), cudaMemcpyDeviceToHost, c->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return HYDRO_ECUDA;
  if (d.status != 0) return (hydro_status)d.status;
  if (g.cfl_limit > 0.0 && nsteps > 0) {
    double vmax;
    std::memcpy(&vmax, &d.vmax_bits, sizeof(vmax));
    if (vmax * g.dt / g.dx > g.cfl_limit) return HYDRO_ECFL;
  }
  return HYDRO_OK;
}

hydro_status hydro_read_fields(hydro_ctx* c, int32_t kind, double* host5) {
  if (!c || !host5 || (kind != HYDRO_PRIMITIVE && kind != HYDRO_CONSERVED)) return HYDRO_EINVAL;
  if (!c->initialized) return HYDRO_ESTATE;
  prof_mark(c, HYDRO_KERNEL_OTHER);
  cudaError_t e = launch_readback(c->cfg.precision, kind, c->U(c->lay.u0), c->staging(), c->n, c->cfg.e_floor,
                                  c->stream);
  prof_mark(c, HYDRO_KERNEL_OTHER);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host5, c->staging(), 5 * c->n * sizeof(double), cudaMemcpyDefault, c->stream);   // host or device
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

hydro_status hydro_get_diag(hydro_ctx* c, hydro_diag* out) {
  if (!c || !out) return HYDRO_EINVAL;
  DevDiag d;
  cudaError_t e = cudaMemcpyAsync(&d, c->diag(), sizeof(d), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return HYDRO_ECUDA;
  std::memset(out, 0, sizeof(*out));
  out->t = c->cfg.t0 + (double)c->steps * c->cfg.dt;
  out->steps = c->steps;
  std::memcpy(&out->max_speed, &d.vmax_bits, sizeof(double));
  out->floor_hits = (int64_t)d.floor_hits;
  out->njet = c->njet;
  for (int j = 0; j < c->njet; ++j) {
    out->dep_E += d.dep[j];
    for (int a = 0; a < 3; ++a) {
      out->dep_M[a] += c->jn[j][a] * d.dep[j];
      out->jet_cell[j][a] = d.cell[j][a];
    }
  }
  for (int j = c->njet; j < kMaxJets; ++j)
    for (int a = 0; a < 3; ++a) out->jet_cell[j][a] = -1;
  out->status = d.status;
  out->check_site = d.check_site;
  out->check_index = d.check_index;
  return HYDRO_OK;
}

hydro_status hydro_profile_enable(hydro_ctx* c, int32_t on) {
  if (!c) return HYDRO_EINVAL;
  prof_clear(c);
  c->profiling = on != 0;
  return HYDRO_OK;
}

hydro_status hydro_profile_query(hydro_ctx* c, int32_t kind, double* total_ms, int64_t* launches) {
  if (!c || kind < 0 || kind >= HYDRO_KERNEL_COUNT) return HYDRO_EINVAL;
  hydro_status s = prof_resolve(c);
  if (s != HYDRO_OK) return s;
  if (total_ms) *total_ms = c->prof.ms[kind];
  if (launches) *launches = c->prof.n[kind];
  return HYDRO_OK;
}

void hydro_destroy(hydro_ctx* c) {
  if (!c) return;
  if (c->stream || c->ws) cudaStreamSynchronize(c->stream);
  prof_clear(c);
  if (c->owns_ws && c->ws) cudaFree(c->ws);
  delete c;
}

const char* hydro_status_string(hydro_status s) {
  switch (s) {
    case HYDRO_OK: return "HYDRO_OK";
    case HYDRO_EINVAL: return "HYDRO_EINVAL: invalid argument or configuration";
    case HYDRO_ENOMEM: return "HYDRO_ENOMEM: device memory";
    case HYDRO_ECUDA: return "HYDRO_ECUDA: CUDA error";
    case HYDRO_EUNPHYSICAL: return "HYDRO_EUNPHYSICAL: NaN or Inf in the state";
    case HYDRO_ECFL: return "HYDRO_ECFL: CFL limit exceeded";
    case HYDRO_ETIMEOUT: return "HYDRO_ETIMEOUT: bounded wait expired";
    case HYDRO_ESTATE: return "HYDRO_ESTATE: call out of order";
    case HYDRO_ECHECK: return "HYDRO_ECHECK: a bounds check of the checked build failed";
    default: return "unknown hydro_status";
  }
}

}  // extern "C"
