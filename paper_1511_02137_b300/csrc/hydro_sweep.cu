// Directional flux sweeps of one RK3 stage (arXiv:1511.02137, Sec. 1, Eqs. 1-3).
//
// A stage evaluates L(U) = -sum_d (Fhat_{i+1/2} - Fhat_{i-1/2})/dx + S and
// combines it with the step's start state.  It runs as three sweeps, one per
// axis, each a tiled kernel with one updated cell per thread:
//
//   phase 0  (FP32-flux y and z sweeps, and the mixed x sweep) start copying
//            the tile's phase-3 operands (accumulator; z: the step state U0)
//            into shared memory: one TMA box each, or per-thread cp.async
//            copies;
//   phase 1  stage a halo-padded tile of cells into shared memory (interior
//            tiles as one TMA box, edge tiles through clamped or wrapped
//            coalesced loads; mixed precision stages the FP32 shadow of the
//            stage state), recover primitives in closed form (the FP64 y and z
//            sweeps read them from the x sweep's cache instead), and keep U,
//            the half physical flux F_d/2 and the spectral radius rho_d of
//            every cell;
//   phase 2  one thread per interface: alpha = max rho_d over the interface's
//            stencil, local Lax-Friedrichs split f_pm = F/2 +- alpha U/2, and
//            component-wise WENO reconstruction of f+ (left-biased) and f-
//            (right-biased, mirrored); Fhat = f+ + f-;
//   phase 3  one thread per cell: the flux difference goes into the
//            right-hand-side accumulator (x: write, y: add; FP32-flux tiles
//            store the box by TMA); the z sweep adds the jet source at the jet
//            cells and writes the stage combination a U0 + b (U + dt L) in
//            storage precision (mixed precision keeps the stage states as FP32
//            increments over U0 in the accumulator: its z sweep forms U0 + delta
//            in FP64 for the next FP32 shadow and, at the last stage, the new
//            state).
//
// Ghost cells are never stored: halo loads clamp the index (outflow,
// zero-gradient) or wrap it (periodic).  The x sweep of each stage counts
// primitive-recovery floors; at the first stage of a step every sweep folds
// its spectral radii into the step's maximum signal speed with a warp
// reduction and one atomic per block.  Element indices are 32-bit (a grid
// holds at most 4e8 cells).
#include <cstdint>
#include <cstring>

#include "hydro.h"
#include "hydro_check.cuh"
#include "hydro_internal.h"
#include "hydro_math.cuh"

namespace hydro {

// Storage type of the state, arithmetic type of the fluxes, and the math
// policy of the flux arithmetic.  Mixed: FP64 storage and RK3 accumulation,
// FP64 for the cancelling part of the primitive recovery, FP32 for the rest.
// kMixedShadow is the mixed precision of single-grid contexts: the sweeps stage
// an FP32 shadow of each stage state (mixed_shadow: the five roundings and
// om = 1 - |M|/E from E^2 - |M|^2 in FP64), written by the z sweep that forms
// the state, so that no staged cell is converted or recovered in FP64 again;
// and the stage states are kept as FP32 increments over the step state U0,
// delta_k = U_k - U0, in the right-hand-side accumulator itself: with a + b = 1
// the stage combination is delta_{k+1} = b delta_k + b dt (L_x + L_y + L_z + S),
// which the x sweep starts (b delta_k + b dt L_x), the y sweep continues and
// the z sweep finishes, forming U_{k+1} = U0 + delta_{k+1} in FP64 for the
// shadow and, at the last stage, as the new FP64 state.  The increments carry
// FP32 accuracy relative to their own size; no FP64 stage state other than U0
// is stored.  Every mixed-precision run (single grid, batch, the adjoint's
// forward) takes this form.
constexpr int kMixedShadow = 3;
template <int PREC> struct Types;
template <> struct Types<HYDRO_FP64> { using Store = double; using Flux = double; using Math = MathD; };
template <> struct Types<HYDRO_FP32> { using Store = float; using Flux = float; using Math = MathF; };
template <> struct Types<kMixedShadow> { using Store = double; using Flux = float; using Math = MathF; };
template <int PREC> constexpr bool kIsMixed = PREC == kMixedShadow;
// Fields of a staged cell as stored: 5, or 6 for the mixed shadow (with om).
template <int PREC> constexpr int kStagedFields = PREC == kMixedShadow ? 6 : 5;

// Tile shape per sweep axis: SEG cells along the sweep axis, LANES lines.  The
// lines of the y and z sweeps run along x so that loads stay coalesced.
// FP64 keeps the longer x tile (fewer recomputed halo cells per FP64-bound
// interface); FP32 and mixed run the x sweep on 32 x 8 tiles, faster when
// instruction issue bounds the kernel.
template <int PREC, int DIR> struct Tile { static constexpr int SEG = 32, LANES = 8; };
template <> struct Tile<HYDRO_FP64, 0> { static constexpr int SEG = 64, LANES = 4; };

constexpr int kThreads = 256;

__device__ __forceinline__ int map_along(int i, int n, int periodic) {
  if (periodic) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// A launch constant in the flux or storage type: the host-rounded FP32 copy or
// the FP64 original.
template <class T>
__device__ __forceinline__ T kconst(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}

// Maximum of two non-negative values.  Non-negative doubles order like their
// bit patterns, so FP64 takes the integer maximum and leaves the FP64 pipe
// (1/64 of the FP32 rate on this part) to the arithmetic.
__device__ __forceinline__ double max_nonneg(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}
__device__ __forceinline__ float max_nonneg(float a, float b) { return fmaxf(a, b); }

// ---- TMA staging (cp.async.bulk.tensor) with an mbarrier, bounded wait

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// 4-D tiled copy (x, y, z, field) of one box into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// 4-D tiled copy of one box from shared memory to global memory (bulk async
// group; the part of the box past the tensor's extent is not written).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
               : "memory");
}
// Commits the issued bulk stores and waits until they have read shared memory.
__device__ __forceinline__ void tma_store_commit_wait_read() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Orders this thread's shared-memory writes before later async-proxy (TMA) reads.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Asynchronous global -> shared copies of B bytes (cp.async, L1-allocating).
template <int B>
__device__ __forceinline__ void cp_async_ca(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(smem)), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The GPU's global nanosecond timer.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the barrier phase for at most limit_ns of global time (try_wait
// itself suspends the thread for a while between checks); false when the limit
// ran out first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, phase))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// Block-wide max of the spectral radius and sum of floor hits, published with
// one atomic each.  Must be reached by every thread of the block.
template <class T>
__device__ __forceinline__ void publish_block(T vmax, unsigned hits, DevDiag* d, bool speed, bool floors) {
  __shared__ T wmax[kThreads / 32];
  __shared__ unsigned whits[kThreads / 32];
  // warp reductions: one redux.sync each for the hit count and, in FP32, for the
  // maximum (vmax >= 0 and never NaN: fmax drops NaN spectral radii, and
  // non-negative floats order like their bit patterns); FP64 maxima by shuffles
  hits = __reduce_add_sync(0xffffffffu, hits);
  if constexpr (sizeof(T) == 4) {
    vmax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(vmax)));
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    wmax[w] = vmax;
    whits[w] = hits;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T mt = T(0);
    unsigned long long h = 0;
    for (int i = 0; i < kThreads / 32; ++i) {
      mt = fmax(mt, wmax[i]);
      h += whits[i];
    }
    const double m = (double)mt;
    // non-negative doubles order like their bit patterns
    if (speed) atomicMax(&d->vmax_bits, (unsigned long long)__double_as_longlong(m));
    if (floors && h) atomicAdd(&d->floor_hits, h);
  }
}

// FP32 flux arithmetic issues fast enough that the phase-3 operands (the
// accumulator of the y and z sweeps and the step state U0) are fetched into
// shared memory asynchronously at the start
// of the tile, so that their latency hides behind phases 1 and 2.  FP64 tiles
// are bound by the FP64 pipe and keep the direct loads (and their occupancy).
// The mixed shadow's x sweep also fetches the accumulator (delta_k).
template <int PREC, int DIR>
struct Prefetch {
  static constexpr bool on = sizeof(typename Types<PREC>::Flux) == 4 && (DIR != 0 || PREC == kMixedShadow);
  static constexpr int rhs = on ? 5 : 0;                      // accumulator fields
  // step-state operands in flux-type words per cell: U0 (FP32, or FP64 in mixed
  // precision)
  static constexpr int state_words = on && DIR == 2 ? (PREC == kMixedShadow ? 10 : 5) : 0;
};

// The sweeps stage interior tiles with one TMA copy (single grids in WENO7 and
// WENO5, whose x tiles are the exception, see stage_by_tma; batches, which run
// WENO7).  FP64 copies
// straight into the tile's U array; FP32 tiles interleave U with F_d/2, so their
// copy lands in a separate staging box that phase 1 reads; the mixed shadow's x
// and y sweeps copy the shadow the same way.  The mixed z tile, which also holds
// U0 in FP64, would lose a resident block per SM to a separate box: its box lands
// on the (U, F_d/2) area instead, which phase 1 fills only after every thread has
// read its staged cells into registers (see kBoxAliased).
template <int PREC, int DIR = 0>
__host__ __device__ constexpr bool tma_staged() {
  return true;
}

// Whether a tile of this sweep stages by TMA.  A box must start at an innermost
// (x) coordinate whose byte offset is a multiple of 16: the x sweep's box starts at
// a0 - G, aligned for WENO7 (G = 4, a0 a multiple of the segment) but not for
// WENO5 (G = 3), whose x tiles therefore stage through plain loads; the y and z
// boxes start at the lane origin l0, a multiple of LANES.
template <int PREC, int ORDER, int DIR>
__host__ __device__ constexpr bool stage_by_tma() {
  return tma_staged<PREC, DIR>() && (ORDER == 7 || DIR != 0);
}

// The staging box of this tile shares the start of the (U, F_d/2) area.
template <int PREC, int DIR>
constexpr bool kBoxAliased = PREC == kMixedShadow && DIR == 2;

// Shared memory of one tile, in units of the flux type (word offsets): U, F_d/2
// (5 fields each) and rho_d per staged cell, 5 numerical fluxes per interface,
// the prefetched phase-3 operands per updated cell, (FP64 WENO7) the neighbour
// differences, and (FP32 with TMA staging) the staging box of 5 fields per staged
// cell.  Areas that a TMA copy writes start on 128-byte boundaries.
template <int PREC, int ORDER, int DIR, int SEG, int LANES>
struct TileLayout {
  using F = typename Types<PREC>::Flux;
  using Store = typename Types<PREC>::Store;
  static constexpr int G = (ORDER == 7) ? 4 : 3, NCS = LANES * (SEG + 2 * G), NIF = LANES * (SEG + 1),
                       NC = LANES * SEG;
  static constexpr int A = 128 / (int)sizeof(F);   // words per 128 bytes
  __host__ __device__ static constexpr int up(int w) { return (w + A - 1) / A * A; }
  static constexpr int pr = up(11 * NCS + 5 * NIF);                      // [5][NC] accumulator
  static constexpr int p0 = pr + Prefetch<PREC, DIR>::rhs * NC;          // [5][NC] U0 (+ [5][NC] U), Store
  static constexpr int delta = p0 + Prefetch<PREC, DIR>::state_words * NC;
  static constexpr int body = delta + ((sizeof(F) == 8 && ORDER == 7) ? 10 * NCS : 0);
  static constexpr int stage = up(body);
  __host__ __device__ static constexpr int words(bool stage_box) {
    if (kBoxAliased<PREC, DIR>) return body;
    return (stage_box && sizeof(F) == 4) ? stage + kStagedFields<PREC> * NCS : body;
  }
};

template <int PREC, int ORDER, int DIR, int SEG, int LANES, bool STAGE = false>
__host__ __device__ constexpr int tile_smem_words() {
  return TileLayout<PREC, ORDER, DIR, SEG, LANES>::words(STAGE);
}

// One tile of a sweep: SEG cells along the sweep axis starting at a0, LANES
// lines starting at l0, in plane `fixed` (z for the x and y sweeps, y for the z
// sweep).  Must be reached by every thread of the block; shared memory is free
// again when it returns.
// The two mbarriers of a block's TMA copies (staging box, phase-3 operands),
// initialised once per block, and the parity of the next phase of each; every
// thread of the block keeps the same copy of the parities.
struct TileBars {
  uint64_t* stage;
  uint64_t* pf;
  unsigned ph_stage, ph_pf;
};

// Initialises the block's mbarriers (one arrival each: the thread that issues the
// copies).  Must be reached by every thread of the block.
__device__ __forceinline__ void init_tile_bars(TileBars& tb) {
  if (threadIdx.x == 0) {
    mbar_init(tb.stage, 1);
    mbar_init(tb.pf, 1);
  }
  __syncthreads();
  tb.ph_stage = 0;
  tb.ph_pf = 0;
}

// A bounded wait for a TMA copy that runs out sets the status word and, when
// given, *late (shared memory); after a second bounded wait for the copy the
// tile finishes on whatever shared memory holds.
template <int PREC, int ORDER, int DIR, bool FINAL, int SEG, int LANES, bool TMA = false>
__device__ __forceinline__ void sweep_tile(const GridArgs& a, const JetStage& jets, int a0, int l0, int fixed,
                                           unsigned char* smem_raw, const SweepMaps* maps = nullptr,
                                           TileBars* tb = nullptr, int* late = nullptr) {
  using Store = typename Types<PREC>::Store;
  using F = typename Types<PREC>::Flux;
  using Math = typename Types<PREC>::Math;
  constexpr int G = (ORDER == 7) ? 4 : 3;   // halo width = half the interface stencil
  constexpr int W = SEG + 2 * G;            // staged cells per line
  constexpr int NCS = LANES * W;            // staged cells
  constexpr int NIF = LANES * (SEG + 1);    // interfaces
  constexpr int NC = LANES * SEG;           // updated cells

  // FP32 flux type: U and F_d/2 of a cell interleaved ([5][NCS] float2), so that
  // one 64-bit load brings both to an interface; FP64: [5][NCS] U then [5][NCS] F_d/2
  constexpr bool IL = sizeof(F) == 4;
  F* sU = reinterpret_cast<F*>(smem_raw);   // [5][NCS] conserved (FP64)
  F* sF = sU + 5 * NCS;                     // [5][NCS] F_d / 2 (FP64)
  float2* sUF = reinterpret_cast<float2*>(smem_raw);   // [5][NCS] (U, F_d/2) (FP32)
  F* sR = sU + 10 * NCS;                    // [NCS]    rho_d
  F* sH = sR + NCS;                         // [5][NIF] numerical flux

  const int nx = a.nx, ny = a.ny, nz = a.nz;
  // 32-bit element indices: a grid holds at most 4e8 cells, so 5 fields stay below 2^32
  const unsigned N = (unsigned)nx * ny * nz;
  const int n_along = DIR == 0 ? nx : (DIR == 1 ? ny : nz);
  const int n_lane = DIR == 0 ? ny : nx;
  auto offset = [&](int along, int lane) -> unsigned {
    if (DIR == 0) return ((unsigned)fixed * ny + lane) * nx + along;
    if (DIR == 1) return ((unsigned)fixed * ny + along) * nx + lane;
    return ((unsigned)along * ny + fixed) * nx + lane;
  };
  // staged cell (lane, s) and interface/cell (lane, j) index maps; consecutive
  // threads walk the contiguous (x) direction in every phase
  auto sidx = [&](int lane, int s) { return DIR == 0 ? lane * W + s : s * LANES + lane; };
  auto hidx = [&](int lane, int j) { return DIR == 0 ? lane * (SEG + 1) + j : j * LANES + lane; };

  // ---------------- phase-3 operands, fetched asynchronously
  const Store* __restrict__ U = static_cast<const Store*>(a.U);
  using PF = Prefetch<PREC, DIR>;
  using TL = TileLayout<PREC, ORDER, DIR, SEG, LANES>;
  F* sPr = reinterpret_cast<F*>(smem_raw) + TL::pr;                          // [5][NC] accumulator
  Store* sP0 = reinterpret_cast<Store*>(reinterpret_cast<F*>(smem_raw) + TL::p0);   // [5][NC] U0
  // every tile shape updates one cell per thread (phase 3 and its operands)
  static_assert(NC == kThreads, "one updated cell per thread");
  // the mixed shadow's z sweep needs U0 at every stage (U_{k+1} = U0 + delta_{k+1}),
  // and its x sweep at the first stage reads no increment (delta_0 = 0)
  constexpr bool SH = PREC == kMixedShadow;
  const bool need_u0 = FINAL && (SH || !a.k.first);
  const bool pf_want = !(SH && DIR == 0 && a.k.first);
  if constexpr (PF::on && TMA) {
    // one thread copies the tile's boxes of cells (the box of an edge tile reaches
    // past the grid and is filled with zeros there, which phase 3 does not read)
    if (threadIdx.x == 0 && pf_want) {
      const unsigned bytes = (unsigned)(5 * NC * sizeof(F) +
                                        (need_u0 ? 5 * NC * sizeof(Store) : 0));
      mbar_expect_tx(tb->pf, bytes);
      if (!a.withhold) {
        const int c0 = DIR == 0 ? a0 : l0, c1 = DIR == 0 ? l0 : (DIR == 1 ? a0 : fixed),
                  c2 = DIR == 2 ? a0 : fixed;
        if (HYDRO_TMA_OK(c0, (int)sizeof(F), c1, c2, false)) tma_load_4d(sPr, &maps->rhs, c0, c1, c2, 0, tb->pf);
        if (need_u0 && HYDRO_TMA_OK(c0, (int)sizeof(Store), c1, c2, false))
          tma_load_4d(sP0, &maps->u0, c0, c1, c2, 0, tb->pf);
      }
    }
  } else if constexpr (PF::on) {
    const F* rhs_in = static_cast<const F*>(a.rhs);
    const Store* U0_in = static_cast<const Store*>(a.U0);
    const int c = threadIdx.x;
    int lane, j;
    if (DIR == 0) { lane = c / SEG; j = c - lane * SEG; }
    else { j = c / LANES; lane = c - j * LANES; }
    const int ga = a0 + j, gl = l0 + lane;
    if (ga < n_along && gl < n_lane && pf_want) {
      const unsigned o = HYDRO_CELL(offset(ga, gl), N, kSiteOperands);
#pragma unroll
      for (int q = 0; q < 5; ++q) cp_async_ca<sizeof(F)>(sPr + q * NC + c, rhs_in + q * N + o);
      if constexpr (FINAL) {
        if (need_u0) {
#pragma unroll
          for (int q = 0; q < 5; ++q) cp_async_ca<sizeof(Store)>(sP0 + q * NC + c, U0_in + q * N + o);
        }
      }
    }
    cp_async_commit();
  }

  // whether a jet deposits into this tile (z sweep), decided once per block and
  // read in phase 3 after the barriers of phases 1 and 2
  __shared__ int sJetFlag;
  int* sJet = &sJetFlag;
  if (FINAL && threadIdx.x == 0) {
    int here = 0;
    for (int jn = 0; jn < jets.n; ++jn) {
      const int* cl = jets.cell[jn];
      if (cl[0] < 0) continue;
      const int jal = DIR == 0 ? cl[0] : (DIR == 1 ? cl[1] : cl[2]);
      const int jln = DIR == 0 ? cl[1] : cl[0];
      const int jfx = DIR == 2 ? cl[1] : cl[2];
      if (jfx == fixed && jal >= a0 && jal < a0 + SEG && jln >= l0 && jln < l0 + LANES) here = 1;
    }
    *sJet = here;
  }

  // ---------------- phase 1: stage cells, primitives, half fluxes, rho
  // a tile whose halo lies inside the grid needs no ghost cells: one TMA box of all
  // 5 fields (6 shadow fields for kMixedShadow)
  bool staged = false;
  F* sStage = kBoxAliased<PREC, DIR> ? reinterpret_cast<F*>(smem_raw)   // [5 or 6][NCS] as copied
                                      : (IL ? reinterpret_cast<F*>(smem_raw) + TL::stage : sU);
  constexpr int NSF = kStagedFields<PREC>;
  if constexpr (TMA && stage_by_tma<PREC, ORDER, DIR>()) {
    static_assert(PREC == kMixedShadow || sizeof(Store) == sizeof(F),
                  "TMA staging copies the stored type into the flux-type tile");
    if (a0 - G >= 0 && a0 + SEG + G <= n_along && l0 + LANES <= n_lane) {
      if (threadIdx.x == 0) {
        mbar_expect_tx(tb->stage, (unsigned)(NSF * NCS * sizeof(F)));
        if (a.withhold) {
          // fault injection: the barrier is armed but no copy is issued
        } else if (DIR == 0) {
          if (HYDRO_TMA_OK(a0 - G, (int)sizeof(F), l0, fixed, false))
            tma_load_4d(sStage, &maps->stage, a0 - G, l0, fixed, 0, tb->stage);
        } else if (DIR == 1) {
          if (HYDRO_TMA_OK(l0, (int)sizeof(F), a0 - G, fixed, false))
            tma_load_4d(sStage, &maps->stage, l0, a0 - G, fixed, 0, tb->stage);
        } else if (HYDRO_TMA_OK(l0, (int)sizeof(F), fixed, a0 - G, false)) {
          tma_load_4d(sStage, &maps->stage, l0, fixed, a0 - G, 0, tb->stage);
        }
      }
      if (!mbar_wait_bounded(tb->stage, tb->ph_stage, a.wait_ns)) {
        atomicCAS(&a.diag->status, 0, (int)HYDRO_ETIMEOUT);
        if (late) *late = 1;
        // the copy may still land: wait once more (bounded) so that none is left
        // in flight into this block's shared memory; a withheld copy never comes
        if (!a.withhold) mbar_wait_bounded(tb->stage, tb->ph_stage, a.wait_ns);
      }
      tb->ph_stage ^= 1u;
      staged = true;
    }
  }
  F vmax = F(0);
  unsigned hits = 0;
  // FP64: the y and z sweeps take v_d, p and rho_d of their staged cells from the x
  // sweep's cache when there is one, and recover nothing (FP32 and mixed tiles
  // recover faster than they would load, and compile without the cache)
  constexpr bool CACHE = PREC == HYDRO_FP64;
  F* __restrict__ Pc = CACHE ? static_cast<F*>(a.P) : nullptr;
  const bool cached = CACHE && DIR != 0 && Pc != nullptr;
  // a thread's staged cells c = threadIdx.x + r kThreads, r < NR; an aliased box is
  // read into registers before the barrier after which phase 1 overwrites it
  constexpr int NR = (NCS + kThreads - 1) / kThreads;
  constexpr bool ALIAS = kBoxAliased<PREC, DIR>;
  float box[ALIAS ? NR : 1][6];
  if constexpr (ALIAS) {
    if (staged) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int c = threadIdx.x + r * kThreads;
        if (c < NCS) {
#pragma unroll
          for (int f = 0; f < 6; ++f) box[r][f] = sStage[f * NCS + c];
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int c = threadIdx.x + r * kThreads;
    if (c >= NCS) break;
    int lane, s;
    if (DIR == 0) { lane = c / W; s = c - lane * W; }
    else { s = c / LANES; lane = c - s * LANES; }
    const int ga = a0 - G + s;
    const int gl = l0 + lane;
    F e, vx, vy, vz, E, Mx, My, Mz, R;
    F v2, rden;   // v^2 and 1/(1 - v^2/3) from the recovery (FP64, FP32)
    F p, vd, rho;
    int hit = 0;
    if constexpr (PREC == kMixedShadow) {
      // the shadow written with the state: FP32 values and om, no FP64 work here
      float om;
      if (ALIAS && staged) {
        E = box[r][0]; Mx = box[r][1]; My = box[r][2]; Mz = box[r][3]; R = box[r][4]; om = box[r][5];
      } else if (staged) {
        E = sStage[c]; Mx = sStage[NCS + c]; My = sStage[2 * NCS + c]; Mz = sStage[3 * NCS + c];
        R = sStage[4 * NCS + c]; om = sStage[5 * NCS + c];
      } else {
        const float* __restrict__ S = a.S;
        const unsigned o =
            HYDRO_CELL(offset(map_along(ga, n_along, a.periodic), gl < n_lane ? gl : n_lane - 1), N, kSiteStaging);
        E = S[o]; Mx = S[N + o]; My = S[2 * N + o]; Mz = S[3 * N + o]; R = S[4 * N + o]; om = S[5 * N + o];
      }
      cons_to_prim_shadow_rho(E, Mx, My, Mz, om, a.k.e_floor_f, e, vx, vy, vz, v2, rden, hit);
    } else if constexpr (CACHE) {
      const unsigned og =
          HYDRO_CELL(offset(map_along(ga, n_along, a.periodic), gl < n_lane ? gl : n_lane - 1), N, kSiteStaging);
      Store Es, Mxs, Mys, Mzs, Rs;
      if (staged) {
        Es = (Store)sStage[c]; Mxs = (Store)sStage[NCS + c]; Mys = (Store)sStage[2 * NCS + c];
        Mzs = (Store)sStage[3 * NCS + c]; Rs = (Store)sStage[4 * NCS + c];
      } else {
        Es = U[og]; Mxs = U[N + og]; Mys = U[2 * N + og]; Mzs = U[3 * N + og]; Rs = U[4 * N + og];
      }
      E = (F)Es; Mx = (F)Mxs; My = (F)Mys; Mz = (F)Mzs; R = (F)Rs;
      if (cached) {
        // cache layout v_y, rho_y, p, v_z, rho_z: the y sweep reads fields 0-2, the z sweep 2-4
        vd = Pc[(DIR == 1 ? 0 : 3) * N + og];
        rho = Pc[(DIR == 1 ? 1 : 4) * N + og];
        p = Pc[2 * N + og];
      } else {
        cons_to_prim_rho<Math>(Es, Mxs, Mys, Mzs, kconst<F>(a.e_floor, a.k.e_floor_f), e, vx, vy, vz, v2, rden, hit);
        if (DIR == 0 && Pc != nullptr && s >= G && s < G + SEG && ga < n_along && gl < n_lane) {
          // this tile's own cells: their primitives for the y and z sweeps of the stage
          Pc[og] = vy;
          Pc[N + og] = spectral_radius_r<Math>(vy, v2, rden);
          Pc[2 * N + og] = e * F(1.0 / 3.0);
          Pc[3 * N + og] = vz;
          Pc[4 * N + og] = spectral_radius_r<Math>(vz, v2, rden);
        }
      }
    } else {
      Store Es, Mxs, Mys, Mzs, Rs;
      if (staged) {
        Es = (Store)sStage[c]; Mxs = (Store)sStage[NCS + c]; Mys = (Store)sStage[2 * NCS + c];
        Mzs = (Store)sStage[3 * NCS + c]; Rs = (Store)sStage[4 * NCS + c];
      } else {
        const unsigned o =
            HYDRO_CELL(offset(map_along(ga, n_along, a.periodic), gl < n_lane ? gl : n_lane - 1), N, kSiteStaging);
        Es = U[o]; Mxs = U[N + o]; Mys = U[2 * N + o]; Mzs = U[3 * N + o]; Rs = U[4 * N + o];
      }
      cons_to_prim_rho<Math>(Es, Mxs, Mys, Mzs, kconst<F>(a.e_floor, a.k.e_floor_f), e, vx, vy, vz, v2, rden, hit);
      E = (F)Es; Mx = (F)Mxs; My = (F)Mys; Mz = (F)Mzs; R = (F)Rs;
    }
    if (!cached) {
      p = e * F(1.0 / 3.0);
      vd = DIR == 0 ? vx : (DIR == 1 ? vy : vz);
      rho = spectral_radius_r<Math>(vd, v2, rden);
    }
    const F Md = DIR == 0 ? Mx : (DIR == 1 ? My : Mz);
    const F Fh[5] = {F(0.5) * Md, F(0.5) * (Mx * vd + (DIR == 0 ? p : F(0))),
                     F(0.5) * (My * vd + (DIR == 1 ? p : F(0))), F(0.5) * (Mz * vd + (DIR == 2 ? p : F(0))),
                     F(0.5) * (R * vd)};
    if constexpr (IL) {
      sUF[0 * NCS + c] = make_float2(E, Fh[0]);
      sUF[1 * NCS + c] = make_float2(Mx, Fh[1]);
      sUF[2 * NCS + c] = make_float2(My, Fh[2]);
      sUF[3 * NCS + c] = make_float2(Mz, Fh[3]);
      sUF[4 * NCS + c] = make_float2(R, Fh[4]);
    } else {
      if (!staged) {
        sU[0 * NCS + c] = E;
        sU[1 * NCS + c] = Mx;
        sU[2 * NCS + c] = My;
        sU[3 * NCS + c] = Mz;
        sU[4 * NCS + c] = R;
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) sF[q * NCS + c] = Fh[q];
    }
    sR[c] = rho;
    if (s >= G && s < G + SEG && ga < n_along && gl < n_lane) {
      vmax = fmax(vmax, rho);
      hits += (unsigned)hit;
    }
  }
  if (a.reduce_speed || a.count_floors) publish_block(vmax, hits, a.diag, a.reduce_speed, a.count_floors);
  __syncthreads();

  // FP64 WENO7: differences of U and F/2 between neighbouring staged cells, once
  // per cell pair; each interface then forms its split-flux differences with one
  // FMA apiece instead of splitting 8 cells and differencing per interface.
  constexpr bool DELTA = sizeof(F) == 8 && ORDER == 7;
  F* sDU = reinterpret_cast<F*>(smem_raw) + TL::delta;   // [5][NCS] U(c+1) - U(c)
  F* sDF = sDU + 5 * NCS;                                 // [5][NCS] F(c+1) - F(c)
  if constexpr (DELTA) {
    for (int c = threadIdx.x; c < NCS; c += kThreads) {
      int lane, s;
      if (DIR == 0) { lane = c / W; s = c - lane * W; }
      else { s = c / LANES; lane = c - s * LANES; }
      if (s + 1 >= W) continue;
      const int cn = sidx(lane, s + 1);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        sDU[q * NCS + c] = sU[q * NCS + cn] - sU[q * NCS + c];
        sDF[q * NCS + c] = sF[q * NCS + cn] - sF[q * NCS + c];
      }
    }
    __syncthreads();
  }

  // ---------------- phase 2: numerical flux at every interface of the tile
  const F eps = kconst<F>(a.k.eps_s, a.k.eps_s_f);
  // numerical flux of components q0 .. q1-1 at the interface left of tile cell j
  // (its stencil is staged cells j .. j + 2G - 1)
  auto flux_at = [&](int lane, int j, int q0, int q1) {
    F alpha = sR[sidx(lane, j)];
#pragma unroll
    for (int t = 1; t < 2 * G; ++t) alpha = max_nonneg(alpha, sR[sidx(lane, j + t)]);
    const F ah = F(0.5) * alpha;
#pragma unroll 1
    for (int q = q0; q < q1; ++q) {
      F u[2 * G], f[2 * G];
#pragma unroll
      for (int t = 0; t < 2 * G; ++t) {
        if constexpr (IL) {
          const float2 uf = sUF[q * NCS + sidx(lane, j + t)];
          u[t] = uf.x;
          f[t] = uf.y;
        } else {
          u[t] = sU[q * NCS + sidx(lane, j + t)];
          f[t] = sF[q * NCS + sidx(lane, j + t)];
        }
      }
      F h;
      if constexpr (ORDER == 7 && sizeof(F) == 4) {
        // lane x: f+ from cells i-3..i+3; lane y: f- mirrored from cells i+4..i-2
        // (scalar FMAs that write the two lanes directly: a packed split would first
        // have to move each cell's values into two different register pairs)
        float2 g[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) g[k] = make_float2(fmaf(ah, u[k], f[k]), fmaf(-ah, u[7 - k], f[7 - k]));
        const float2 hh = weno7_pair(g[0], g[1], g[2], g[3], g[4], g[5], g[6], eps);
        h = hh.x + hh.y;
      } else if constexpr (ORDER == 7) {
        // FP64: f+ from cells i-3..i+3 and the negated mirrored f- from cells i+4..i-2,
        // their differences from the neighbour differences; one division for both
        F dp[6], dm[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          dp[k] = fma(ah, sDU[q * NCS + sidx(lane, j + k)], sDF[q * NCS + sidx(lane, j + k)]);
          dm[k] = fma(-ah, sDU[q * NCS + sidx(lane, j + 6 - k)], sDF[q * NCS + sidx(lane, j + 6 - k)]);
        }
        h = weno7_sum_d1(fma(ah, u[3], f[3]), dp, fma(ah, u[4], -f[4]), dm, eps);
      } else if constexpr (sizeof(F) == 4) {
        // WENO5, FP32: lane x f+ from cells i-2..i+2, lane y f- mirrored from i+3..i-1
        float2 g[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) g[k] = make_float2(fmaf(ah, u[k], f[k]), fmaf(-ah, u[5 - k], f[5 - k]));
        const float2 hh = weno5_pair(g[0], g[1], g[2], g[3], g[4], eps);
        h = hh.x + hh.y;
      } else {
        h = weno5<F>(fma(ah, u[0], f[0]), fma(ah, u[1], f[1]), fma(ah, u[2], f[2]), fma(ah, u[3], f[3]),
                     fma(ah, u[4], f[4]), eps) +
            weno5<F>(fma(-ah, u[5], f[5]), fma(-ah, u[4], f[4]), fma(-ah, u[3], f[3]), fma(-ah, u[2], f[2]),
                     fma(-ah, u[1], f[1]), eps);
      }
      sH[q * NIF + hidx(lane, j)] = h;
    }
  };
  // the left faces of the tile's cells, all components, then the right face of
  // each line split into single-component tasks so that no thread does two
  // whole interfaces while the block waits at the barrier
  {
    const int it = threadIdx.x;
    int lane, j;
    if (DIR == 0) { lane = it / SEG; j = it - lane * SEG; }
    else { j = it / LANES; lane = it - j * LANES; }
    flux_at(lane, j, 0, 5);
  }
  for (int t = threadIdx.x; t < 5 * LANES; t += kThreads) {
    const int q = t / LANES, lane = t - q * LANES;
    flux_at(lane, SEG, q, q + 1);
  }
  __syncthreads();

  // ---------------- phase 3: flux difference, source, stage combination
  const bool jets_here = FINAL && *sJet != 0;
  // FP32-flux x and y tiles with tensor maps write their accumulator values into
  // shared memory and store them as one TMA box: the x sweep into the staged-cell
  // area (free once phase 2 is done), the y sweep into the prefetched accumulator.
  // (The z sweep keeps per-thread stores of the stage result: a TMA store there
  // measured slower, 0.546 vs 0.534 ms per FP32 launch at 256^3.)
  constexpr bool TST = TMA && IL && !FINAL;
  F* sOut = reinterpret_cast<F*>(smem_raw);   // [5][NC] (x sweep)
  F* __restrict__ rhs = static_cast<F*>(a.rhs);
  const F inv_dx = kconst<F>(a.inv_dx, a.k.inv_dx_f);
  bool bad = false;
  if constexpr (PF::on && TMA) {
    if (pf_want) {
      if (!mbar_wait_bounded(tb->pf, tb->ph_pf, a.wait_ns)) {
        atomicCAS(&a.diag->status, 0, (int)HYDRO_ETIMEOUT);
        if (late) *late = 1;
        if (!a.withhold) mbar_wait_bounded(tb->pf, tb->ph_pf, a.wait_ns);   // as for the staging copy
      }
      tb->ph_pf ^= 1u;
    }
  } else if constexpr (PF::on) {
    cp_async_wait_all();   // each thread reads only its own copies
  }
  {
    const int c = threadIdx.x;
    int lane, j;
    if (DIR == 0) { lane = c / SEG; j = c - lane * SEG; }
    else { j = c / LANES; lane = c - j * LANES; }
    const int ga = a0 + j, gl = l0 + lane;
    if (ga < n_along && gl < n_lane) {
      const unsigned o = HYDRO_CELL(offset(ga, gl), N, kSiteUpdate);
      const int h0 = hidx(lane, j), h1 = hidx(lane, j + 1);
      F L[5];
      if constexpr (SH) {
        // the mixed shadow accumulates the stage increment b dt L (x: on top of b delta_k),
        // one product with b dt / dx per flux difference
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          L[q] = (sH[q * NIF + h0] - sH[q * NIF + h1]) * a.k.bdt_dx_f;
          if (DIR == 0 && !a.k.first) L[q] = fmaf(a.k.b_f, PF::on ? sPr[q * NC + c] : rhs[q * N + o], L[q]);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 5; ++q) L[q] = -(sH[q * NIF + h1] - sH[q * NIF + h0]) * inv_dx;
      }
      if (!FINAL) {
        if constexpr (TST && DIR == 0) {
#pragma unroll
          for (int q = 0; q < 5; ++q) sOut[q * NC + c] = L[q];
        } else if constexpr (TST) {
#pragma unroll
          for (int q = 0; q < 5; ++q) sPr[q * NC + c] += L[q];
        } else if (DIR == 0) {
#pragma unroll
          for (int q = 0; q < 5; ++q) rhs[q * N + o] = L[q];
        } else {
#pragma unroll
          for (int q = 0; q < 5; ++q) rhs[q * N + o] = (PF::on ? sPr[q * NC + c] : rhs[q * N + o]) + L[q];
        }
      } else {
        // the stage's right-hand side in the flux type
        F Lq[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) Lq[q] = (PF::on ? sPr[q * NC + c] : rhs[q * N + o]) + L[q];
        if (jets_here) {
          const int gx = DIR == 0 ? ga : gl;
          const int gy = DIR == 1 ? ga : (DIR == 0 ? gl : fixed);
          const int gz = DIR == 2 ? ga : fixed;
          for (int jn = 0; jn < jets.n; ++jn) {
            const int* cl = jets.cell[jn];
            if (cl[0] != gx || cl[1] != gy || cl[2] != gz) continue;
            // Eq. 3 at the temperature of this cell, deposited as in Eq. 2
            double e;
            int hit = 0;
            if constexpr (SH) {
              // the stage state's recovery from its shadow (FP32 e: the source enters in FP32)
              const float* S = a.S;
              float ef, vxf, vyf, vzf, v2f, rdf;
              cons_to_prim_shadow_rho(S[o], S[N + o], S[2 * N + o], S[3 * N + o], S[5 * N + o], a.k.e_floor_f, ef,
                                      vxf, vyf, vzf, v2f, rdf, hit);
              e = ef;
            } else {
              double vx, vy, vz;
              cons_to_prim<MathD>((double)U[o], (double)U[N + o], (double)U[2 * N + o], (double)U[3 * N + o],
                                   a.e_floor, e, vx, vy, vz, hit);
            }
            const double T = temperature(e, a.src.t4coef);
            const double S0 = (a.src.rad * T * T * T * jets.ell[jn] + a.src.coll * T * T) * a.src.inv_vol;
            const double Sw = SH ? a.b * a.dt * S0 : S0;   // the mixed shadow accumulates b dt S
            Lq[0] += (F)Sw;
            Lq[1] += (F)(jets.dir[jn][0] * Sw);
            Lq[2] += (F)(jets.dir[jn][1] * Sw);
            Lq[3] += (F)(jets.dir[jn][2] * Sw);
            a.diag->dep[jn] += a.src.wdt_vol * S0;
            a.diag->cell[jn][0] = gx;
            a.diag->cell[jn][1] = gy;
            a.diag->cell[jn][2] = gz;
          }
        }
        // U0 and Uout alias at the last stage (in-place update of the step state)
        const Store* U0 = static_cast<const Store*>(a.U0);
        Store* Uout = static_cast<Store*>(a.Uout);
        const Store dt = kconst<Store>(a.dt, a.k.dt_f), ca = kconst<Store>(a.a, a.k.a_f), cb = kconst<Store>(a.b, a.k.b_f);
        // FP32: the finite test runs once on the sum of the five results (NaN and
        // infinities propagate into it; a finite sum of physical values cannot overflow)
        float chk = 0.0f;
        Store outv[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          Store out;
          if constexpr (SH) {
            // Lq = delta_{k+1} (FP32); U_{k+1} = U0 + delta_{k+1} in FP64.  Before the
            // last stage the increment goes back into the accumulator for the next x sweep.
            out = sP0[q * NC + c] + f2d(Lq[q]);
            if (!Uout) rhs[q * N + o] = Lq[q];
          } else {
            // the cell's own state is staged already
            const Store u = IL ? (Store)sUF[q * NCS + sidx(lane, j + G)].x : (Store)sU[q * NCS + sidx(lane, j + G)];
            const Store l = Lq[q];
            out = a.k.first ? u + dt * l : ca * (PF::on ? sP0[q * NC + c] : U0[q * N + o]) + cb * (u + dt * l);
          }
          // (the mixed shadow path tests its FP32 increments: U0 is finite, as the
          // result of the previous step or of a checked initial state)
          if constexpr (sizeof(Store) == 4) chk += out;
          else if constexpr (SH) chk += Lq[q];
          else bad |= !finite_bits(out);
          if (PREC != kMixedShadow || Uout) Uout[q * N + o] = out;   // (the shadow stores U only at stage 3)
          outv[q] = out;
        }
        if constexpr (sizeof(Store) == 4 || SH) bad |= !finite_bits(chk);
        if constexpr (PREC == kMixedShadow) {
          // the shadow of the new state, for the sweeps that stage it next
          float sh[6];
          mixed_shadow(outv[0], outv[1], outv[2], outv[3], outv[4], a.e_floor, sh);
          float* __restrict__ So = a.Sout;
#pragma unroll
          for (int q = 0; q < 6; ++q) So[q * N + o] = sh[q];
        }
      }
    }
  }
  if (FINAL && bad) atomicCAS(&a.diag->status, 0, (int)HYDRO_EUNPHYSICAL);
  if constexpr (TST) {
    // the tile's results leave as one box (clipped at the grid's edge)
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      if (DIR == 0) {
        if (HYDRO_TMA_OK(a0, (int)sizeof(F), l0, fixed, true)) tma_store_4d(&maps->rhs, sOut, a0, l0, fixed, 0);
      } else if (HYDRO_TMA_OK(l0, (int)sizeof(F), a0, fixed, true)) {
        tma_store_4d(&maps->rhs, sPr, l0, a0, fixed, 0);
      }
      tma_store_commit_wait_read();
    }
  }
}

// One single-grid sweep tile per block.
template <int PREC, int ORDER, int DIR, bool FINAL, bool TMA>
__device__ __forceinline__ void sweep_block(const SweepArgs& a, const SweepMaps& maps) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar, bar_pf;
  TileBars tb{&bar, &bar_pf, 0u, 0u};
  if constexpr (TMA) init_tile_bars(tb);
  constexpr int SEG = Tile<PREC, DIR>::SEG, LANES = Tile<PREC, DIR>::LANES;
  int a0, l0;
  if (DIR == 0) {
    a0 = blockIdx.x * SEG; l0 = blockIdx.y * LANES;
  } else {
    l0 = blockIdx.x * LANES; a0 = blockIdx.y * SEG;
  }
  sweep_tile<PREC, ORDER, DIR, FINAL, SEG, LANES, TMA>(a, a.jets, a0, l0, blockIdx.z, smem_raw, &maps, &tb);
}

template <int PREC, int ORDER, int DIR, bool FINAL, bool TMA>
__global__ void __launch_bounds__(kThreads) sweep_kernel(const SweepArgs a, const __grid_constant__ SweepMaps maps) {
  sweep_block<PREC, ORDER, DIR, FINAL, TMA>(a, maps);
}

// The FP32 and mixed-shadow z sweeps held to 40 registers (six blocks of 256
// threads per SM); left alone they take 46-48 and five blocks.  The other sweeps
// stay at or below 40 by themselves; FP64 tiles are limited by shared memory
// first.
template <int PREC, int ORDER, bool TMA>
__global__ void __launch_bounds__(kThreads, 6) sweep_kernel_z6(const SweepArgs a, const __grid_constant__ SweepMaps maps) {
  sweep_block<PREC, ORDER, 2, true, TMA>(a, maps);
}

// Resident blocks per SM the batched kernels' register budget is held to: six
// FP32-flux blocks (40 registers, as the single-grid sweeps), three FP64 blocks
// (their shared memory admits no more).
template <int PREC>
__host__ __device__ constexpr int batch_min_blocks() { return PREC == HYDRO_FP64 ? 3 : 6; }

// Batched sweep over the tile list of all grids of the ensemble: one block per
// tile, or persistent blocks that walk the list (tile t, t + gridDim.x, ...).  A
// tile is two int4 in the list, (event, a0, l0, fixed) and its grid's (nx, ny,
// nz, first cell), read together, so that a block starts its tile after one
// global read; persistent blocks keep the next two tiles' entries in flight
// (cp.async) while they work.
template <int PREC, int DIR, bool FINAL, int SEG, int LANES, bool TMA>
__global__ void __launch_bounds__(kThreads, batch_min_blocks<PREC>()) batch_sweep_kernel(const BatchArgs b) {
  using Store = typename Types<PREC>::Store;
  using F = typename Types<PREC>::Flux;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the tile's grid arguments live in shared memory (one thread fills them): held in
  // registers across the tile they would cost the persistent kernel occupancy
  __shared__ GridArgs g;
  __shared__ __align__(16) int4 tdq[3][2];   // entries of this tile and the next two
  __shared__ int4 td;
  __shared__ __align__(8) uint64_t bar, bar_pf;
  __shared__ int sLate;   // a wait of this block ran out (set once, never cleared)
  TileBars tb{&bar, &bar_pf, 0u, 0u};
  const int G = (int)gridDim.x;
  auto fetch = [&](int q, int t) {
    cp_async_ca<16>(&tdq[q][0], &b.tiles[2 * (size_t)t]);
    cp_async_ca<16>(&tdq[q][1], &b.tiles[2 * (size_t)t + 1]);
  };
  if (threadIdx.x == 0) {
    sLate = 0;
    // the fields every tile shares
    g.periodic = b.periodic;
    g.inv_dx = b.inv_dx;
    g.dt = b.dt;
    g.a = b.a;
    g.b = b.b;
    g.e_floor = b.e_floor;
    g.eps = b.eps;
    g.reduce_speed = b.reduce_speed;
    g.count_floors = b.count_floors;
    g.wait_ns = b.wait_ns;
    g.withhold = b.withhold;
    g.check_tighten = b.check_tighten;
    g.src = b.src;
    g.k = b.k;
    const int t0 = blockIdx.x;
    if (t0 < b.ntiles) fetch(0, t0);
    if (t0 + G < b.ntiles) fetch(1, t0 + G);
    cp_async_commit();
  }
  if constexpr (TMA) init_tile_bars(tb);   // (its barrier also orders the writes above)
  else __syncthreads();
  int it = 0;
  for (int t = blockIdx.x; t < b.ntiles; t += G, ++it) {
    if (threadIdx.x == 0) {
      cp_async_wait_all();   // this tile's entries (and the next tile's)
      const int q = it % 3;
      if (t + 2 * G < b.ntiles) {
        fetch((it + 2) % 3, t + 2 * G);
        cp_async_commit();
      }
      td = tdq[q][0];
      const int4 gd = tdq[q][1];
      const size_t cell0 = (unsigned)gd.w;
      const size_t off = 5 * cell0;   // element offset of the grid's 5 fields
      g.U = static_cast<const Store*>(b.U) + off;
      g.U0 = static_cast<const Store*>(b.U0) + off;
      g.Uout = b.Uout ? static_cast<Store*>(b.Uout) + off : nullptr;
      g.rhs = static_cast<F*>(b.rhs) + off;
      g.P = b.P ? static_cast<F*>(b.P) + off : nullptr;
      g.diag = b.diags + td.x;
      g.nx = gd.x;
      g.ny = gd.y;
      g.nz = gd.z;
      g.S = b.S ? b.S + 6 * cell0 : nullptr;   // the grid's shadow block: 6 fields of its cells
      g.Sout = b.Sout ? b.Sout + 6 * cell0 : nullptr;
    }
    __syncthreads();
    const int4 tile = td;
    sweep_tile<PREC, 7, DIR, FINAL, SEG, LANES, TMA>(g, b.jets[tile.x], tile.y, tile.z, tile.w, smem_raw,
                                                     TMA ? b.maps + tile.x : nullptr, &tb, &sLate);
    // the next tile overwrites shared memory, partly by TMA: order this tile's
    // generic-proxy writes before the async proxy's
    if constexpr (TMA) fence_proxy_async_smem();
    __syncthreads();
    // after a wait that ran out the barriers' phases are no longer known: the
    // whole block stops (the step reports HYDRO_ETIMEOUT).  sLate is written only
    // inside a tile, so every thread reads the same value here.
    if (sLate) break;
  }
  // a block that stopped early may still have copies of the next tiles in flight
  if (threadIdx.x == 0) cp_async_wait_all();
}

__global__ void reset_vmax_kernel(DevDiag* d, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i].vmax_bits = 0ull;
}

template <int PREC, int ORDER, int DIR, bool TMA>
static auto pick_sweep_kernel() {
  if constexpr ((PREC == HYDRO_FP32 || PREC == kMixedShadow) && DIR == 2) return sweep_kernel_z6<PREC, ORDER, TMA>;
  else return sweep_kernel<PREC, ORDER, DIR, DIR == 2, TMA>;
}

template <int PREC, int ORDER, int DIR>
static cudaError_t launch_one(const SweepArgs& a, cudaStream_t s, const SweepMaps* maps) {
  using F = typename Types<PREC>::Flux;
  constexpr int SEG = Tile<PREC, DIR>::SEG, LANES = Tile<PREC, DIR>::LANES;
  // tensor maps serve the staging copy (FP64, FP32, the mixed shadow's x and y
  // sweeps), and the phase-3 operands and results of FP32-flux tiles (FP32, mixed)
  constexpr bool kStage = stage_by_tma<PREC, ORDER, DIR>();
  constexpr bool kMapsUsed = kStage || sizeof(F) == 4;
  constexpr size_t smem = sizeof(F) * (size_t)tile_smem_words<PREC, ORDER, DIR, SEG, LANES>();
  constexpr size_t smem_tma = sizeof(F) * (size_t)tile_smem_words<PREC, ORDER, DIR, SEG, LANES, kStage>();
  dim3 grid;
  if (DIR == 0) grid = dim3((a.nx + SEG - 1) / SEG, (a.ny + LANES - 1) / LANES, a.nz);
  else if (DIR == 1) grid = dim3((a.nx + LANES - 1) / LANES, (a.ny + SEG - 1) / SEG, a.nz);
  else grid = dim3((a.nx + LANES - 1) / LANES, (a.nz + SEG - 1) / SEG, a.ny);
  if (kMapsUsed && maps) {
    auto kern = pick_sweep_kernel<PREC, ORDER, DIR, kMapsUsed>();
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tma);
    if (err != cudaSuccess) return err;
    kern<<<grid, kThreads, smem_tma, s>>>(a, *maps);
    return cudaGetLastError();
  }
  auto kern = pick_sweep_kernel<PREC, ORDER, DIR, false>();
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  SweepMaps none;
  memset(&none, 0, sizeof(none));
  kern<<<grid, kThreads, smem, s>>>(a, none);
  return cudaGetLastError();
}

template <int PREC, int ORDER>
static cudaError_t launch_dir(int dir, const SweepArgs& a, cudaStream_t s, const SweepMaps* t) {
  switch (dir) {
    case 0: return launch_one<PREC, ORDER, 0>(a, s, t);
    case 1: return launch_one<PREC, ORDER, 1>(a, s, t);
    default: return launch_one<PREC, ORDER, 2>(a, s, t);
  }
}

template <int PREC>
static cudaError_t launch_order(int order, int dir, const SweepArgs& a, cudaStream_t s, const SweepMaps* t) {
  return order == 5 ? launch_dir<PREC, 5>(dir, a, s, t) : launch_dir<PREC, 7>(dir, a, s, t);
}

LaunchConst derive_constants(const GridArgs& g, int order) {
  LaunchConst k;
  // the indicators are used in scaled form (720/781 beta for WENO7, 12/13 beta for WENO5)
  k.eps_s = (order == 7 ? kW7EpsScale : kW5EpsScale) * g.eps;
  k.eps_s_f = (float)k.eps_s;
  k.inv_dx_f = (float)g.inv_dx;
  k.dt_f = (float)g.dt;
  k.a_f = (float)g.a;
  k.b_f = (float)g.b;
  k.e_floor_f = (float)g.e_floor;
  k.bdt_dx_f = (float)(g.b * g.dt * g.inv_dx);
  k.first = g.a == 0.0;
  return k;
}

cudaError_t launch_sweep(int precision, int order, int dir, const SweepArgs& args, cudaStream_t s,
                         const SweepMaps* tmap) {
  SweepArgs a = args;
  a.k = derive_constants(a, order);
  if (a.wait_ns == 0) a.wait_ns = kDefaultWaitNs;
  switch (precision) {
    case HYDRO_FP64: return launch_order<HYDRO_FP64>(order, dir, a, s, tmap);
    case HYDRO_FP32: return launch_order<HYDRO_FP32>(order, dir, a, s, tmap);
    default:
      // mixed precision stages the shadows of its stage states
      return a.S ? launch_order<kMixedShadow>(order, dir, a, s, tmap) : cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------- tensor maps


// The tile shape of a single-grid sweep (Tile<PREC, DIR>) at run time.
static void tile_shape(int precision, int d, int& seg, int& lanes) {
  auto pick = [&](auto prec_tag) {
    constexpr int P = decltype(prec_tag)::value;
    if (d == 0) { seg = Tile<P, 0>::SEG; lanes = Tile<P, 0>::LANES; }
    else if (d == 1) { seg = Tile<P, 1>::SEG; lanes = Tile<P, 1>::LANES; }
    else { seg = Tile<P, 2>::SEG; lanes = Tile<P, 2>::LANES; }
  };
  if (precision == HYDRO_FP64) pick(std::integral_constant<int, HYDRO_FP64>());
  else if (precision == HYDRO_FP32) pick(std::integral_constant<int, HYDRO_FP32>());
  else pick(std::integral_constant<int, HYDRO_MIXED>());
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_entry() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return nullptr;
  }
  return reinterpret_cast<EncodeTiled>(fn);
}

// The maps of one grid for the three stages and axes, with tile shapes seg[d] x lanes[d];
// shadows (mixed precision, may be NULL) give the staging boxes of the FP32 shadows.
// order: the WENO order, whose halo of G = (order + 1) / 2 cells on each side sets
// the staging boxes (none for the x sweep of WENO5, see stage_by_tma).
static bool encode_grid(EncodeTiled encode, int precision, void* const bufs[3], void* rhs, int nx, int ny, int nz,
                        const int seg[3], const int lanes[3], SweepMaps maps[3][3],
                        void* const shadows[3] = nullptr, int order = 7) {
  const int halo2 = order + 1;   // staged cells beyond a tile's segment
  const size_t es = precision == HYDRO_FP32 ? 4 : 8;   // stored type
  const size_t fs = precision == HYDRO_FP64 ? 8 : 4;   // flux type
  // a 4-D (x, y, z, field) map of one array of box[3] fields with elements of `size` bytes
  auto enc = [&](CUtensorMap* m, void* base, size_t size, const cuuint32_t box[4]) {
    const cuuint64_t dim[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)box[3]};
    const cuuint64_t stride[3] = {(cuuint64_t)nx * size, (cuuint64_t)nx * ny * size, (cuuint64_t)nx * ny * nz * size};
    for (int k = 0; k < 3; ++k)
      if (stride[k] % 16 != 0) return false;
    if ((box[0] * size) % 16 != 0 || reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = size == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return encode(m, dt, 4, base, dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  // box of a tile's staged cells (W = SEG + 8 along the axis) or updated cells (SEG)
  auto box_of = [&](int d, int ln, int along, cuuint32_t box[4]) {
    box[3] = 5;
    if (d == 0) { box[0] = along; box[1] = ln; box[2] = 1; }
    else if (d == 1) { box[0] = ln; box[1] = along; box[2] = 1; }
    else { box[0] = ln; box[1] = 1; box[2] = along; }
  };
  std::memset(maps, 0, 9 * sizeof(SweepMaps));
  for (int st = 0; st < 3; ++st)
    for (int d = 0; d < 3; ++d) {
      cuuint32_t box[4];
      const bool staged = order == 7 || d != 0;
      if (precision == HYDRO_MIXED && !shadows) {
        return false;                  // mixed precision stages shadows only
      } else if (precision != HYDRO_MIXED && staged) {   // staging box of the stage state
        box_of(d, lanes[d], seg[d] + halo2, box);
        if (!enc(&maps[st][d].stage, bufs[st], es, box)) return false;
      } else if (staged) {             // staging box of the stage state's FP32 shadow (6 fields)
        box_of(d, lanes[d], seg[d] + halo2, box);
        box[3] = 6;
        if (!enc(&maps[st][d].stage, shadows[st], 4, box)) return false;
      }
      if (precision != HYDRO_FP64) {   // phase-3 operand and result boxes
        box_of(d, lanes[d], seg[d], box);
        if (!enc(&maps[st][d].rhs, rhs, fs, box)) return false;
        if (d == 2) {
          if (!enc(&maps[st][d].u0, bufs[0], es, box)) return false;
        }
      }
    }
  return true;
}

bool encode_sweep_tmaps(int precision, int order, void* const bufs[3], void* rhs, int nx, int ny, int nz,
                        SweepMaps maps[3][3], void* const shadows[3]) {
  if (order != 7 && order != 5) return false;
  EncodeTiled encode = encode_entry();
  if (!encode) return false;
  int seg[3], lanes[3];
  for (int d = 0; d < 3; ++d) tile_shape(precision, d, seg[d], lanes[d]);
  return encode_grid(encode, precision, bufs, rhs, nx, ny, nz, seg, lanes, maps, shadows, order);
}

bool encode_batch_tmaps(int precision, void* const bufs[3], void* rhs, int nev, const int32_t* dims,
                        const size_t* off, const int variant[3], SweepMaps* maps, void* const shadows[3]) {
  EncodeTiled encode = encode_entry();
  if (!encode) return false;
  const size_t es = precision == HYDRO_FP32 ? 4 : 8, fs = precision == HYDRO_FP64 ? 8 : 4;
  int seg[3], lanes[3];
  seg[0] = kTileSegX[variant[0]];
  lanes[0] = kTileLanesX[variant[0]];
  for (int d = 1; d < 3; ++d) {
    seg[d] = kTileSegYZ[variant[d]];
    lanes[d] = kTileLanesYZ[variant[d]];
  }
  for (int e = 0; e < nev; ++e) {
    void* eb[3];
    void* es6[3];
    for (int k = 0; k < 3; ++k) {
      eb[k] = static_cast<char*>(bufs[k]) + off[e] * es;
      es6[k] = shadows ? static_cast<char*>(shadows[k]) + off[e] / 5 * 6 * sizeof(float) : nullptr;
    }
    SweepMaps m[3][3];
    if (!encode_grid(encode, precision, eb, static_cast<char*>(rhs) + off[e] * fs, dims[3 * e], dims[3 * e + 1],
                     dims[3 * e + 2], seg, lanes, m, shadows ? es6 : nullptr))
      return false;
    for (int st = 0; st < 3; ++st)
      for (int d = 0; d < 3; ++d) maps[(size_t)(st * 3 + d) * nev + e] = m[st][d];
  }
  return true;
}

// ---------------------------------------------------------------- batched launches

// Batched tiles with tensor maps take the same TMA paths as single-grid tiles.
template <int PREC, int DIR, int SEG, int LANES, bool TMA>
static constexpr size_t batch_smem() {
  using F = typename Types<PREC>::Flux;
  return sizeof(F) * (size_t)tile_smem_words<PREC, 7, DIR, SEG, LANES, TMA && tma_staged<PREC, DIR>()>();
}

template <int PREC, int DIR, int SEG, int LANES, bool TMA>
static auto batch_kernel_ptr() {
  return batch_sweep_kernel<PREC, DIR, DIR == 2, SEG, LANES, TMA>;
}

template <int PREC, int DIR, int V, bool TMA>
static cudaError_t batch_launch_vt(const BatchArgs& a, int grid, cudaStream_t s) {
  constexpr int SEG = DIR == 0 ? kTileSegX[V] : kTileSegYZ[V];
  constexpr int LANES = DIR == 0 ? kTileLanesX[V] : kTileLanesYZ[V];
  constexpr size_t smem = batch_smem<PREC, DIR, SEG, LANES, TMA>();
  auto kern = batch_kernel_ptr<PREC, DIR, SEG, LANES, TMA>();
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int PREC, int DIR, int V>
static cudaError_t batch_launch_v(const BatchArgs& a, int grid, cudaStream_t s) {
  return a.maps ? batch_launch_vt<PREC, DIR, V, true>(a, grid, s) : batch_launch_vt<PREC, DIR, V, false>(a, grid, s);
}

template <int PREC, int DIR, int V, bool TMA>
static int batch_occupancy_vt() {
  constexpr int SEG = DIR == 0 ? kTileSegX[V] : kTileSegYZ[V];
  constexpr int LANES = DIR == 0 ? kTileLanesX[V] : kTileLanesYZ[V];
  constexpr size_t smem = batch_smem<PREC, DIR, SEG, LANES, TMA>();
  auto kern = batch_kernel_ptr<PREC, DIR, SEG, LANES, TMA>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kThreads, smem) != cudaSuccess) return 0;
  return n;
}

template <int PREC, int DIR, int V>
static int batch_occupancy_v(bool tma) {
  return tma ? batch_occupancy_vt<PREC, DIR, V, true>() : batch_occupancy_vt<PREC, DIR, V, false>();
}

template <int PREC, int DIR>
static cudaError_t batch_launch_dir(int variant, const BatchArgs& a, int grid, cudaStream_t s) {
  switch (variant) {
    case 0: return batch_launch_v<PREC, DIR, 0>(a, grid, s);
    case 1: return batch_launch_v<PREC, DIR, 1>(a, grid, s);
    default: return batch_launch_v<PREC, DIR, 2>(a, grid, s);
  }
}

template <int PREC, int DIR>
static int batch_occupancy_dir(int variant, bool tma) {
  switch (variant) {
    case 0: return batch_occupancy_v<PREC, DIR, 0>(tma);
    case 1: return batch_occupancy_v<PREC, DIR, 1>(tma);
    default: return batch_occupancy_v<PREC, DIR, 2>(tma);
  }
}

template <int PREC>
static cudaError_t batch_launch_prec(int dir, int variant, const BatchArgs& a, int grid, cudaStream_t s) {
  switch (dir) {
    case 0: return batch_launch_dir<PREC, 0>(variant, a, grid, s);
    case 1: return batch_launch_dir<PREC, 1>(variant, a, grid, s);
    default: return batch_launch_dir<PREC, 2>(variant, a, grid, s);
  }
}

template <int PREC>
static int batch_occupancy_prec(int dir, int variant, bool tma) {
  switch (dir) {
    case 0: return batch_occupancy_dir<PREC, 0>(variant, tma);
    case 1: return batch_occupancy_dir<PREC, 1>(variant, tma);
    default: return batch_occupancy_dir<PREC, 2>(variant, tma);
  }
}

cudaError_t launch_batch_sweep(int precision, int dir, int variant, const BatchArgs& args, int grid, cudaStream_t s) {
  if (grid <= 0 || args.ntiles <= 0) return cudaSuccess;
  BatchArgs a = args;
  if (a.wait_ns == 0) a.wait_ns = kDefaultWaitNs;
  GridArgs g;
  g.inv_dx = a.inv_dx;
  g.dt = a.dt;
  g.a = a.a;
  g.b = a.b;
  g.e_floor = a.e_floor;
  g.eps = a.eps;
  a.k = derive_constants(g, 7);
  // batches of mixed precision always carry shadows (the mixed shadow kernels)
  switch (precision) {
    case HYDRO_FP64: return batch_launch_prec<HYDRO_FP64>(dir, variant, a, grid, s);
    case HYDRO_FP32: return batch_launch_prec<HYDRO_FP32>(dir, variant, a, grid, s);
    default: return batch_launch_prec<kMixedShadow>(dir, variant, a, grid, s);
  }
}

int batch_sweep_blocks_per_sm(int precision, int dir, int variant, bool tma) {
  switch (precision) {
    case HYDRO_FP64: return batch_occupancy_prec<HYDRO_FP64>(dir, variant, tma);
    case HYDRO_FP32: return batch_occupancy_prec<HYDRO_FP32>(dir, variant, tma);
    default: return batch_occupancy_prec<kMixedShadow>(dir, variant, tma);
  }
}

cudaError_t launch_reset_vmax(DevDiag* diags, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  reset_vmax_kernel<<<(n + 127) / 128, 128, 0, s>>>(diags, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- initial state and read-back

// Eq. 1 with p = e/3: E = (e+p) gamma^2 - p, M^i = (e+p) gamma u^i, R = n gamma,
// gamma = sqrt(1 + u.u).  Rejects e < 0 and non-finite input.
template <class Store>
__global__ void init_kernel(int kind, const double* __restrict__ st, Store* __restrict__ U, size_t n,
                            DevDiag* diag) {
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double f0 = st[i], f1 = st[n + i], f2 = st[2 * n + i], f3 = st[3 * n + i], f4 = st[4 * n + i];
    bad |= !(isfinite(f0) && isfinite(f1) && isfinite(f2) && isfinite(f3) && isfinite(f4));
    double E, Mx, My, Mz, R;
    if (kind == HYDRO_PRIMITIVE) {
      bad |= !(f0 >= 0.0);
      const double p = f0 / 3.0, w = f0 + p;
      const double g2 = 1.0 + (f1 * f1 + f2 * f2 + f3 * f3);
      const double g = sqrt(g2);
      E = w * g2 - p;
      Mx = w * g * f1;
      My = w * g * f2;
      Mz = w * g * f3;
      R = f4 * g;
    } else {
      E = f0; Mx = f1; My = f2; Mz = f3; R = f4;
    }
    U[i] = (Store)E;
    U[n + i] = (Store)Mx;
    U[2 * n + i] = (Store)My;
    U[3 * n + i] = (Store)Mz;
    U[4 * n + i] = (Store)R;
  }
  if (bad) atomicExch(&diag->bad_input, 1);
}

template <class Store>
__global__ void readback_kernel(int kind, const Store* __restrict__ U, double* __restrict__ st, size_t n,
                                double e_floor) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double E = U[i], Mx = U[n + i], My = U[2 * n + i], Mz = U[3 * n + i], R = U[4 * n + i];
    if (kind == HYDRO_CONSERVED) {
      st[i] = E; st[n + i] = Mx; st[2 * n + i] = My; st[3 * n + i] = Mz; st[4 * n + i] = R;
    } else {
      double e, vx, vy, vz;
      int hit = 0;
      cons_to_prim<MathD>(E, Mx, My, Mz, e_floor, e, vx, vy, vz, hit);
      const double v2 = vx * vx + vy * vy + vz * vz;
      const double ig = sqrt(1.0 - v2);   // 1/gamma
      const double g = 1.0 / ig;
      st[i] = e; st[n + i] = g * vx; st[2 * n + i] = g * vy; st[3 * n + i] = g * vz; st[4 * n + i] = R * ig;
    }
  }
}

__global__ void shadow_kernel(const double* __restrict__ U, float* __restrict__ S, size_t n, double e_floor) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float sh[6];
    mixed_shadow(U[i], U[n + i], U[2 * n + i], U[3 * n + i], U[4 * n + i], e_floor, sh);
#pragma unroll
    for (int q = 0; q < 6; ++q) S[q * n + i] = sh[q];
  }
}

static unsigned grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b < 148 * 32 ? (b > 0 ? b : 1) : 148 * 32);
}

cudaError_t launch_init(int precision, int kind, const double* staging, void* U, size_t n, DevDiag* diag,
                        cudaStream_t s) {
  if (precision == HYDRO_FP32)
    init_kernel<float><<<grid_for(n), 256, 0, s>>>(kind, staging, static_cast<float*>(U), n, diag);
  else
    init_kernel<double><<<grid_for(n), 256, 0, s>>>(kind, staging, static_cast<double*>(U), n, diag);
  return cudaGetLastError();
}

cudaError_t launch_shadow(const double* U, float* S, size_t n, double e_floor, cudaStream_t s) {
  shadow_kernel<<<grid_for(n), 256, 0, s>>>(U, S, n, e_floor);
  return cudaGetLastError();
}

cudaError_t launch_readback(int precision, int kind, const void* U, double* staging, size_t n, double e_floor,
                            cudaStream_t s) {
  if (precision == HYDRO_FP32)
    readback_kernel<float><<<grid_for(n), 256, 0, s>>>(kind, static_cast<const float*>(U), staging, n, e_floor);
  else
    readback_kernel<double><<<grid_for(n), 256, 0, s>>>(kind, static_cast<const double*>(U), staging, n, e_floor);
  return cudaGetLastError();
}

}  // namespace hydro
