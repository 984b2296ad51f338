// Batched ensembles: many grids of uneven sizes advanced together.
//
// Each sweep of each RK3 stage is one persistent launch that walks the tile
// list of every grid in the ensemble (hydro_sweep.cu, batch_sweep_kernel), so
// small and large grids share the GPU without one launch per grid.  A call to
// hydro_batch_step records the launches of up to kJetChunk steps into one
// CUDA graph (captured once per chunk length and replayed), with the jet cells
// of every grid, step and stage precomputed on the host in FP64 and uploaded
// before the replay.  hydro_batch_autotune times the tile shapes each sweep
// kernel is compiled for on the ensemble itself and keeps the fastest per axis.
// When every grid meets the TMA layout rules, each grid's tensor maps for the
// chosen tile shapes sit in the workspace and the persistent kernels stage,
// fetch and store through them as the single-grid sweeps do.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "hydro.h"
#include "hydro_internal.h"

using namespace hydro;

namespace {

constexpr size_t kAlign = 256;
constexpr int kJetChunk = 64;   // steps per captured graph

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// nx, ny, nz of cfg are ignored (dims give the grids); the batched kernels are
// compiled for WENO7 only.
bool config_ok(const hydro_config* c) { return config_valid(c, kCheckWorkspace) && c->weno_order == 7; }

// Every grid within the single-grid index limit, and the ensemble within the
// 32-bit cell offsets of the tile list.
bool dims_ok(int32_t nev, const int32_t* dims) {
  if (nev < 1 || !dims) return false;
  double total = 0.0;
  for (int e = 0; e < nev; ++e) {
    const int32_t* d = dims + 3 * e;
    if (d[0] < 1 || d[1] < 1 || d[2] < 1) return false;
    if ((double)d[0] * d[1] * d[2] > 4.0e8) return false;
    total += (double)d[0] * d[1] * d[2];
  }
  return total <= 4.0e9;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Tiles of one grid for sweep axis dir with tile shape variant v, two int4 each:
// (event, a0, l0, fixed) and the grid's (nx, ny, nz, first cell), so that a block
// finds everything about its tile in one 32-byte read (see batch_sweep_kernel).
void append_tiles(std::vector<int4>& t, int e, int nx, int ny, int nz, int dir, int v, size_t cell0) {
  const int4 grid = make_int4(nx, ny, nz, (int)(unsigned)cell0);
  auto add = [&](int a0, int l0, int f) {
    t.push_back(make_int4(e, a0, l0, f));
    t.push_back(grid);
  };
  if (dir == 0) {
    const int seg = kTileSegX[v], lanes = kTileLanesX[v];
    for (int z = 0; z < nz; ++z)
      for (int ly = 0; ly < ceil_div(ny, lanes); ++ly)
        for (int ax = 0; ax < ceil_div(nx, seg); ++ax) add(ax * seg, ly * lanes, z);
  } else {
    const int seg = kTileSegYZ[v], lanes = kTileLanesYZ[v];
    const int nalong = dir == 1 ? ny : nz, nfixed = dir == 1 ? nz : ny;
    for (int f = 0; f < nfixed; ++f)
      for (int aa = 0; aa < ceil_div(nalong, seg); ++aa)
        for (int lx = 0; lx < ceil_div(nx, lanes); ++lx) add(aa * seg, lx * lanes, f);
  }
}

size_t max_tiles(int32_t nev, const int32_t* dims, int dir) {
  size_t best = 0;
  for (int v = 0; v < kBatchVariants; ++v) {
    std::vector<int4> t;
    for (int e = 0; e < nev; ++e) append_tiles(t, e, dims[3 * e], dims[3 * e + 1], dims[3 * e + 2], dir, v, 0);
    best = std::max(best, t.size());
  }
  return best;
}

struct BLayout {
  size_t cells = 0;
  size_t u0 = 0, u1 = 0, u2 = 0, rhs = 0, prim = 0, diags = 0, events = 0, tiles[3] = {0, 0, 0}, jets = 0, maps = 0,
         total = 0;
  size_t tile_cap[3] = {0, 0, 0};
  size_t s[3] = {0, 0, 0};   // mixed precision: the FP32 shadows [6][cells] of the three stage states
};

BLayout layout_for(const hydro_config& c, int32_t nev, const int32_t* dims) {
  BLayout L;
  for (int e = 0; e < nev; ++e) L.cells += (size_t)dims[3 * e] * dims[3 * e + 1] * dims[3 * e + 2];
  const size_t store = c.precision == HYDRO_FP32 ? 4 : 8, flux = c.precision == HYDRO_FP64 ? 8 : 4;
  const size_t state = align_up(5 * L.cells * store);
  L.u1 = L.u0 + state;
  L.u2 = L.u1 + state;   // u1 .. u2 end: 5 N doubles of host-transfer staging for any one grid
  L.rhs = L.u2 + state;
  L.prim = L.rhs + align_up(5 * L.cells * flux);   // FP64: primitives cached by the x sweep, laid out as rhs
  L.diags = L.prim + (c.precision == HYDRO_FP64 ? align_up(5 * L.cells * flux) : 0);
  L.events = L.diags + align_up((size_t)nev * sizeof(DevDiag));
  size_t off = L.events + align_up((size_t)nev * sizeof(BatchEvent));
  for (int d = 0; d < 3; ++d) {
    L.tile_cap[d] = max_tiles(nev, dims, d);
    L.tiles[d] = off;
    off += align_up(L.tile_cap[d] * sizeof(int4));
  }
  L.jets = off;
  off += align_up((size_t)kJetChunk * 3 * nev * sizeof(JetStage));
  L.maps = off;   // tensor maps [stage][axis][event]
  off += align_up((size_t)9 * nev * sizeof(SweepMaps));
  for (int k = 0; k < 3; ++k) {
    L.s[k] = off;
    if (c.precision == HYDRO_MIXED) off += align_up(6 * L.cells * sizeof(float));
  }
  L.total = off;
  return L;
}

struct HostJet {
  double x0[3], n[3], t_start;
};

}  // namespace

struct hydro_batch {
  hydro_config cfg;
  int nev = 0;
  std::vector<int32_t> dims;
  std::vector<size_t> off;
  BLayout lay;
  char* ws = nullptr;
  bool owns_ws = false;
  cudaStream_t user = nullptr;
  cudaStream_t cs = nullptr;   // internal stream (capturable)
  int sms = 0;
  int variant[3] = {0, 0, 0};
  int per_tile[3] = {1, 1, 1};   // 1: one block per tile; 0: persistent (blocks per SM x SMs)
  int ntiles[3] = {0, 0, 0};
  int grid[3] = {0, 0, 0};
  bool tma = false;   // tensor maps of the current tile shapes are uploaded
  std::vector<std::vector<HostJet>> jets;
  std::vector<char> initialized;
  int64_t steps = 0;
  cudaGraphExec_t exec = nullptr;
  int exec_steps = 0;
  std::vector<JetStage> jet_host;
  double last_ms[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  char* at(size_t o) { return ws + o; }
  DevDiag* diags() { return reinterpret_cast<DevDiag*>(ws + lay.diags); }
  size_t store() const { return cfg.precision == HYDRO_FP32 ? 4 : 8; }
  float* shadow(int k) { return cfg.precision == HYDRO_MIXED ? reinterpret_cast<float*>(ws + lay.s[k]) : nullptr; }
  size_t flux() const { return cfg.precision == HYDRO_FP64 ? 8 : 4; }
};

namespace {

void drop_graph(hydro_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->exec_steps = 0;
}

// Uploads the tile list and the tensor maps of the current variants and sizes the
// persistent grids.
hydro_status set_tiles(hydro_batch* b) {
  {
    std::vector<SweepMaps> maps((size_t)9 * b->nev);
    void* bufs[3] = {b->at(b->lay.u0), b->at(b->lay.u1), b->at(b->lay.u2)};
    void* shadows[3] = {b->shadow(0), b->shadow(1), b->shadow(2)};
    b->tma = encode_batch_tmaps(b->cfg.precision, bufs, b->at(b->lay.rhs), b->nev, b->dims.data(), b->off.data(),
                                b->variant, maps.data(), b->cfg.precision == HYDRO_MIXED ? shadows : nullptr);
    if (b->tma && cudaMemcpyAsync(b->at(b->lay.maps), maps.data(), maps.size() * sizeof(SweepMaps),
                                  cudaMemcpyHostToDevice, b->cs) != cudaSuccess)
      return HYDRO_ECUDA;
    // the host copy must outlive the asynchronous copy.  No launch of this batch is
    // in flight while the maps are rewritten (every entry point synchronizes the
    // stream before it returns), and the upload completes before the next launch,
    // whose TMA copies read the maps after that launch boundary.
    if (cudaStreamSynchronize(b->cs) != cudaSuccess) return HYDRO_ECUDA;
  }
  for (int d = 0; d < 3; ++d) {
    std::vector<int4> t;
    for (int e = 0; e < b->nev; ++e)
      append_tiles(t, e, b->dims[3 * e], b->dims[3 * e + 1], b->dims[3 * e + 2], d, b->variant[d], b->off[e] / 5);
    if (t.size() > b->lay.tile_cap[d]) return HYDRO_EINVAL;
    if (cudaMemcpyAsync(b->at(b->lay.tiles[d]), t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, b->cs) !=
        cudaSuccess)
      return HYDRO_ECUDA;
    b->ntiles[d] = (int)(t.size() / 2);
    const int per_sm = batch_sweep_blocks_per_sm(b->cfg.precision, d, b->variant[d], b->tma);
    if (per_sm <= 0) return HYDRO_ECUDA;
    b->grid[d] = b->per_tile[d] ? b->ntiles[d]
                                : (int)std::min<long long>((long long)per_sm * b->sms, (long long)b->ntiles[d]);
  }
  drop_graph(b);
  return cudaStreamSynchronize(b->cs) == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

BatchArgs base_args(hydro_batch* b) {
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  const hydro_config& g = b->cfg;
  a.events = reinterpret_cast<const BatchEvent*>(b->at(b->lay.events));
  a.periodic = g.boundary == HYDRO_PERIODIC;
  a.rhs = b->at(b->lay.rhs);
  a.P = g.precision == HYDRO_FP64 ? b->at(b->lay.prim) : nullptr;
  a.diags = b->diags();
  a.inv_dx = 1.0 / g.dx;
  a.dt = g.dt;
  a.e_floor = g.e_floor;
  a.eps = g.weno_eps;
  a.wait_ns = wait_limit_ns(g);
  a.withhold = g.test_withhold_copies;
  a.check_tighten = g.test_check_tighten;
  a.src = source_coef(g);
  return a;
}

// Jet cell at time t (host FP64, no contraction): floor(x/dx + N/2) per axis of
// x = x0 + n (t - t_start); nothing before t_start or outside the grid.
void fill_jet_stage(const hydro_batch* b, int e, double t, JetStage& js) {
  std::memset(&js, 0, sizeof(js));
  const auto& J = b->jets[e];
  const int N[3] = {b->dims[3 * e], b->dims[3 * e + 1], b->dims[3 * e + 2]};
  js.n = (int)J.size();
  for (int j = 0; j < js.n; ++j) {
    jet_cell_at(J[j].x0, J[j].n, J[j].t_start, t, b->cfg.dx, N, js.cell[j], &js.ell[j]);
    for (int a = 0; a < 3; ++a) js.dir[j][a] = J[j].n[a];
  }
}


// Launches (or records, under capture) `n` steps whose jets sit at chunk rows 0..n-1.
cudaError_t issue_steps(hydro_batch* b, int n) {
  const size_t sb = b->store();
  void* U[3] = {b->at(b->lay.u0), b->at(b->lay.u1), b->at(b->lay.u2)};
  BatchArgs a = base_args(b);
  a.U0 = U[0];
  const double vol = b->cfg.dx * b->cfg.dx * b->cfg.dx;
  const JetStage* jt = reinterpret_cast<const JetStage*>(b->at(b->lay.jets));
  (void)sb;
  cudaError_t err = cudaSuccess;
  for (int s = 0; s < n && err == cudaSuccess; ++s) {
    err = launch_reset_vmax(b->diags(), b->nev, b->cs);
    for (int st = 0; st < 3 && err == cudaSuccess; ++st) {
      a.U = U[st];
      a.Uout = st == 2 ? U[0] : U[st + 1];
      if (b->cfg.precision == HYDRO_MIXED) {
        // stage states as FP32 increments over U0 in the accumulator (see hydro_step)
        a.U = U[0];
        a.Uout = st == 2 ? U[0] : nullptr;
        a.S = b->shadow(st);
        a.Sout = b->shadow(st == 2 ? 0 : st + 1);
      }
      a.a = kRK3A[st];
      a.b = kRK3B[st];
      a.src.wdt_vol = b->cfg.dt * kRK3W[st] * vol;
      a.jets = jt + ((size_t)s * 3 + st) * b->nev;
      a.reduce_speed = st == 0;
      for (int d = 0; d < 3 && err == cudaSuccess; ++d) {
        a.tiles = reinterpret_cast<const int4*>(b->at(b->lay.tiles[d]));
        a.maps = b->tma ? reinterpret_cast<const SweepMaps*>(b->at(b->lay.maps)) + (size_t)(st * 3 + d) * b->nev
                        : nullptr;
        a.ntiles = b->ntiles[d];
        a.count_floors = d == 0;
        err = launch_batch_sweep(b->cfg.precision, d, b->variant[d], a, b->grid[d], b->cs);
      }
    }
  }
  return err;
}

bool all_initialized(const hydro_batch* b) {
  for (char c : b->initialized)
    if (!c) return false;
  return true;
}

}  // namespace

extern "C" {

hydro_status hydro_batch_workspace_size(const hydro_config* cfg, int32_t nevents, const int32_t* dims,
                                        size_t* bytes) {
  if (!config_ok(cfg) || !dims_ok(nevents, dims) || !bytes) return HYDRO_EINVAL;
  *bytes = layout_for(*cfg, nevents, dims).total;
  return HYDRO_OK;
}

hydro_status hydro_batch_create(const hydro_config* cfg, int32_t nevents, const int32_t* dims, hydro_batch** out) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  if (!config_ok(cfg) || !dims_ok(nevents, dims)) return HYDRO_EINVAL;
  hydro_batch* b = new (std::nothrow) hydro_batch;
  if (!b) return HYDRO_ENOMEM;
  b->cfg = *cfg;
  b->nev = nevents;
  b->dims.assign(dims, dims + 3 * nevents);
  b->lay = layout_for(*cfg, nevents, dims);
  b->user = static_cast<cudaStream_t>(cfg->cuda_stream);
  b->jets.resize(nevents);
  b->initialized.assign(nevents, 0);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return HYDRO_ECUDA;
  }
  if (cfg->workspace) {
    if (cfg->workspace_bytes < b->lay.total) {
      hydro_batch_destroy(b);
      return HYDRO_ENOMEM;
    }
    b->ws = static_cast<char*>(cfg->workspace);
  } else {
    if (cudaMalloc(&b->ws, b->lay.total) != cudaSuccess) {
      cudaGetLastError();
      hydro_batch_destroy(b);
      return HYDRO_ENOMEM;
    }
    b->owns_ws = true;
  }
  std::vector<BatchEvent> ev(nevents);
  size_t off = 0;
  for (int e = 0; e < nevents; ++e) {
    ev[e].nx = dims[3 * e];
    ev[e].ny = dims[3 * e + 1];
    ev[e].nz = dims[3 * e + 2];
    ev[e].pad = 0;
    ev[e].off = off;
    b->off.push_back(off);
    off += 5 * (size_t)ev[e].nx * ev[e].ny * ev[e].nz;
  }
  if (cudaStreamSynchronize(b->user) != cudaSuccess ||
      cudaMemcpyAsync(b->at(b->lay.events), ev.data(), ev.size() * sizeof(BatchEvent), cudaMemcpyHostToDevice,
                      b->cs) != cudaSuccess ||
      cudaMemsetAsync(b->diags(), 0, (size_t)nevents * sizeof(DevDiag), b->cs) != cudaSuccess) {
    hydro_batch_destroy(b);
    return HYDRO_ECUDA;
  }
  hydro_status st = set_tiles(b);
  if (st != HYDRO_OK) {
    hydro_batch_destroy(b);
    return st;
  }
  *out = b;
  return HYDRO_OK;
}

hydro_status hydro_batch_set_initial(hydro_batch* b, int32_t event, int32_t kind, const double* host5) {
  if (!b || event < 0 || event >= b->nev || !host5 || (kind != HYDRO_PRIMITIVE && kind != HYDRO_CONSERVED))
    return HYDRO_EINVAL;
  const size_t n = (size_t)b->dims[3 * event] * b->dims[3 * event + 1] * b->dims[3 * event + 2];
  double* staging = reinterpret_cast<double*>(b->at(b->lay.u1));
  DevDiag* d = b->diags() + event;
  cudaError_t e = cudaStreamSynchronize(b->user);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(DevDiag), b->cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(staging, host5, 5 * n * sizeof(double), cudaMemcpyDefault, b->cs);
  if (e == cudaSuccess)
    e = launch_init(b->cfg.precision, kind, staging, b->at(b->lay.u0) + b->off[event] * b->store(), n, d, b->cs);
  if (e == cudaSuccess && b->cfg.precision == HYDRO_MIXED)
    e = launch_shadow(reinterpret_cast<const double*>(b->at(b->lay.u0)) + b->off[event],
                      b->shadow(0) + b->off[event] / 5 * 6, n, b->cfg.e_floor, b->cs);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, &d->bad_input, sizeof(int), cudaMemcpyDeviceToHost, b->cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->cs);
  if (e != cudaSuccess) return HYDRO_ECUDA;
  b->initialized[event] = bad ? 0 : 1;
  if (bad) return HYDRO_EINVAL;
  b->steps = 0;
  return HYDRO_OK;
}

hydro_status hydro_batch_add_jet(hydro_batch* b, int32_t event, const double x0[3], const double dir[3],
                                 double t_start, int32_t* jet_id) {
  if (!b || event < 0 || event >= b->nev || !x0 || !dir || !std::isfinite(t_start)) return HYDRO_EINVAL;
  auto& J = b->jets[event];
  if ((int)J.size() >= kMaxJets) return HYDRO_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(x0[a]) || !std::isfinite(dir[a])) return HYDRO_EINVAL;
  const double len = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (!(len > 0.0) || !std::isfinite(len)) return HYDRO_EINVAL;
  HostJet h;
  for (int a = 0; a < 3; ++a) {
    h.x0[a] = x0[a];
    h.n[a] = dir[a] / len;
  }
  h.t_start = t_start;
  J.push_back(h);
  if (jet_id) *jet_id = (int32_t)J.size() - 1;
  return HYDRO_OK;
}

hydro_status hydro_batch_set_tiles(hydro_batch* b, const int32_t variant[3]) {
  if (!b || !variant) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (variant[d] < 0 || variant[d] >= kBatchVariants) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d) b->variant[d] = variant[d];
  return set_tiles(b);
}

hydro_status hydro_batch_set_launch(hydro_batch* b, const int32_t per_tile[3]) {
  if (!b || !per_tile) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (per_tile[d] != 0 && per_tile[d] != 1) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d) b->per_tile[d] = per_tile[d];
  return set_tiles(b);
}

hydro_status hydro_batch_get_tuning(hydro_batch* b, int32_t variant[3], int32_t per_tile[3]) {
  if (!b) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d) {
    if (variant) variant[d] = b->variant[d];
    if (per_tile) per_tile[d] = b->per_tile[d];
  }
  return HYDRO_OK;
}

hydro_status hydro_batch_autotune(hydro_batch* b, int32_t variant_out[3], double ms_out[9]) {
  if (!b) return HYDRO_EINVAL;
  if (!all_initialized(b)) return HYDRO_ESTATE;
  if (cudaStreamSynchronize(b->user) != cudaSuccess) return HYDRO_ECUDA;
  // stage-1 sweeps on the current state, writing only scratch (accumulator and U1); no jets
  JetStage* jt = reinterpret_cast<JetStage*>(b->at(b->lay.jets));
  if (cudaMemsetAsync(jt, 0, (size_t)b->nev * sizeof(JetStage), b->cs) != cudaSuccess) return HYDRO_ECUDA;
  BatchArgs a = base_args(b);
  a.U = a.U0 = b->at(b->lay.u0);
  a.Uout = b->at(b->lay.u1);
  if (b->cfg.precision == HYDRO_MIXED) {   // stage 1 writes the increment and the shadow of U1 only
    a.Uout = nullptr;
    a.S = b->shadow(0);
    a.Sout = b->shadow(1);
  }
  a.a = 0.0;
  a.b = 1.0;
  a.jets = jt;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HYDRO_ECUDA;
  hydro_status status = HYDRO_OK;
  // each tile shape with both launch forms: one block per tile, and persistent blocks
  for (int d = 0; d < 3 && status == HYDRO_OK; ++d) {
    double best = 1e300;
    int best_v = 0, best_m = 1;
    for (int v = 0; v < kBatchVariants && status == HYDRO_OK; ++v) {
      b->last_ms[3 * d + v] = 1e300;
      for (int m = 1; m >= 0 && status == HYDRO_OK; --m) {
        b->variant[d] = v;
        b->per_tile[d] = m;
        status = set_tiles(b);
        if (status != HYDRO_OK) break;
        a.tiles = reinterpret_cast<const int4*>(b->at(b->lay.tiles[d]));
        a.ntiles = b->ntiles[d];
        // stage 1 of a step: the maps of stage 0 for this axis
        a.maps = b->tma ? reinterpret_cast<const SweepMaps*>(b->at(b->lay.maps)) + (size_t)d * b->nev : nullptr;
        double ms_min = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
          cudaEventRecord(e0, b->cs);
          if (launch_batch_sweep(b->cfg.precision, d, v, a, b->grid[d], b->cs) != cudaSuccess) {
            status = HYDRO_ECUDA;
            break;
          }
          cudaEventRecord(e1, b->cs);
          float ms = 0.f;
          if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            status = HYDRO_ECUDA;
            break;
          }
          if (rep > 0) ms_min = std::min(ms_min, (double)ms);
        }
        b->last_ms[3 * d + v] = std::min(b->last_ms[3 * d + v], ms_min);
        if (ms_min < best) {
          best = ms_min;
          best_v = v;
          best_m = m;
        }
      }
    }
    b->variant[d] = best_v;
    b->per_tile[d] = best_m;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != HYDRO_OK) return status;
  status = set_tiles(b);
  if (status != HYDRO_OK) return status;
  // the timing launches may have touched the diagnostics: clear the per-step fields
  for (int e = 0; e < b->nev; ++e) {
    DevDiag* d = b->diags() + e;
    if (cudaMemsetAsync(&d->vmax_bits, 0, sizeof(unsigned long long) * 2, b->cs) != cudaSuccess ||
        cudaMemsetAsync(&d->status, 0, sizeof(int), b->cs) != cudaSuccess)
      return HYDRO_ECUDA;
  }
  if (cudaStreamSynchronize(b->cs) != cudaSuccess) return HYDRO_ECUDA;
  if (variant_out)
    for (int d = 0; d < 3; ++d) variant_out[d] = b->variant[d];
  if (ms_out)
    for (int i = 0; i < 9; ++i) ms_out[i] = b->last_ms[i];
  return HYDRO_OK;
}

hydro_status hydro_batch_step(hydro_batch* b, int32_t nsteps) {
  NvtxRange call("hydro_batch_step");
  if (!b || nsteps < 0) return HYDRO_EINVAL;
  if (!all_initialized(b)) return HYDRO_ESTATE;
  if (cudaStreamSynchronize(b->user) != cudaSuccess) return HYDRO_ECUDA;
  int done = 0;
  while (done < nsteps) {
    const int n = std::min(kJetChunk, nsteps - done);
    // jet cells of every grid at every stage time of this chunk
    b->jet_host.resize((size_t)n * 3 * b->nev);
    for (int s = 0; s < n; ++s)
      for (int st = 0; st < 3; ++st) {
        const double t = b->cfg.t0 + ((double)(b->steps + s) + kRK3C[st]) * b->cfg.dt;
        for (int e = 0; e < b->nev; ++e) fill_jet_stage(b, e, t, b->jet_host[((size_t)s * 3 + st) * b->nev + e]);
      }
    if (cudaMemcpyAsync(b->at(b->lay.jets), b->jet_host.data(), b->jet_host.size() * sizeof(JetStage),
                        cudaMemcpyHostToDevice, b->cs) != cudaSuccess)
      return HYDRO_ECUDA;
    if (!b->exec || b->exec_steps != n) {
      drop_graph(b);
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HYDRO_ECUDA;
      cudaError_t err = issue_steps(b, n);
      cudaError_t end = cudaStreamEndCapture(b->cs, &graph);
      if (err != cudaSuccess || end != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return HYDRO_ECUDA;
      }
      err = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (err != cudaSuccess) {
        b->exec = nullptr;
        return HYDRO_ECUDA;
      }
      b->exec_steps = n;
    }
    if (cudaGraphLaunch(b->exec, b->cs) != cudaSuccess) return HYDRO_ECUDA;
    b->steps += n;
    done += n;
  }
  std::vector<DevDiag> d(b->nev);
  if (cudaMemcpyAsync(d.data(), b->diags(), d.size() * sizeof(DevDiag), cudaMemcpyDeviceToHost, b->cs) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->cs) != cudaSuccess)
    return HYDRO_ECUDA;
  for (int e = 0; e < b->nev; ++e)
    if (d[e].status != 0) return (hydro_status)d[e].status;
  if (b->cfg.cfl_limit > 0.0 && nsteps > 0)
    for (int e = 0; e < b->nev; ++e) {
      double vmax;
      std::memcpy(&vmax, &d[e].vmax_bits, sizeof(vmax));
      if (vmax * b->cfg.dt / b->cfg.dx > b->cfg.cfl_limit) return HYDRO_ECFL;
    }
  return HYDRO_OK;
}

hydro_status hydro_batch_read_fields(hydro_batch* b, int32_t event, int32_t kind, double* host5) {
  if (!b || event < 0 || event >= b->nev || !host5 || (kind != HYDRO_PRIMITIVE && kind != HYDRO_CONSERVED))
    return HYDRO_EINVAL;
  if (!b->initialized[event]) return HYDRO_ESTATE;
  const size_t n = (size_t)b->dims[3 * event] * b->dims[3 * event + 1] * b->dims[3 * event + 2];
  double* staging = reinterpret_cast<double*>(b->at(b->lay.u1));
  cudaError_t e = cudaStreamSynchronize(b->user);
  if (e == cudaSuccess)
    e = launch_readback(b->cfg.precision, kind, b->at(b->lay.u0) + b->off[event] * b->store(), staging, n,
                        b->cfg.e_floor, b->cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host5, staging, 5 * n * sizeof(double), cudaMemcpyDefault, b->cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->cs);
  return e == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

hydro_status hydro_batch_get_diag(hydro_batch* b, int32_t event, hydro_diag* out) {
  if (!b || event < 0 || event >= b->nev || !out) return HYDRO_EINVAL;
  DevDiag d;
  cudaError_t e = cudaMemcpyAsync(&d, b->diags() + event, sizeof(d), cudaMemcpyDeviceToHost, b->cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->cs);
  if (e != cudaSuccess) return HYDRO_ECUDA;
  std::memset(out, 0, sizeof(*out));
  out->t = b->cfg.t0 + (double)b->steps * b->cfg.dt;
  out->steps = b->steps;
  std::memcpy(&out->max_speed, &d.vmax_bits, sizeof(double));
  out->floor_hits = (int64_t)d.floor_hits;
  const auto& J = b->jets[event];
  out->njet = (int32_t)J.size();
  for (int j = 0; j < HYDRO_MAX_JETS; ++j)
    for (int a = 0; a < 3; ++a) out->jet_cell[j][a] = j < out->njet ? d.cell[j][a] : -1;
  for (int j = 0; j < out->njet; ++j) {
    out->dep_E += d.dep[j];
    for (int a = 0; a < 3; ++a) out->dep_M[a] += J[j].n[a] * d.dep[j];
  }
  out->status = d.status;
  out->check_site = d.check_site;
  out->check_index = d.check_index;
  return HYDRO_OK;
}

void hydro_batch_destroy(hydro_batch* b) {
  if (!b) return;
  if (b->cs) cudaStreamSynchronize(b->cs);
  drop_graph(b);
  if (b->owns_ws && b->ws) cudaFree(b->ws);
  if (b->cs) cudaStreamDestroy(b->cs);
  delete b;
}

}  // extern "C"
