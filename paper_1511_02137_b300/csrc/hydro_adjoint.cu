// Adjoint (reverse mode) of the RK3-WENO7 step with jet sources, and a
// cone-energy observable with gradients with respect to k_rad, k_coll and the
// initial energy density (checkpointed every k steps, recomputed in reverse).
// Two precisions, as the forward: FP64 throughout, or mixed (FP64 states,
// stage combinations and adjoint accumulation; FP32 flux arithmetic and its
// vector-Jacobian products; E^2 - |M|^2 of the recovery in FP64).  The forward
// and the recomputation run the step exactly as hydro_step does (the same sweep
// kernels and tensor maps; in mixed precision the stage states are FP32
// increments over the FP64 step state and the sweeps stage their FP32 shadows),
// so the gradient is that of the step the context API computes.
//
// The vector-Jacobian product of the right-hand side L(U) = -div F + S runs as
// three sweeps (x, y, z), like the forward.  A tile gathers, for each of its
// cells, every contribution of the interfaces whose stencils contain the cell
// (so the result is deterministic and needs no atomics): it recomputes alpha,
// the split fluxes and both WENO7 reconstructions of the SEG + 8 interfaces that
// touch its SEG cells, differentiates them in reverse (hydro_adjoint_math.cuh),
// and chains the per-cell adjoints through the half flux F_d/2, the spectral
// radius and the primitive recovery.  The derivative of alpha = max rho is
// split equally among the stencil cells that tie for the maximum (to 1e-12
// relative), the symmetric subgradient.  The z sweep adds the adjoint of the jet
// source of Eqs. 2-3 and accumulates dJ/dk_rad and dJ/dk_coll.  The mixed reverse
// sweeps read the shadows the forward wrote for each stage state.  Outflow
// boundaries only: a clamped ghost hands its adjoint to the edge cell.  The
// backward recomputes the next segment's states from its checkpoint on a side
// stream while the main stream reverses the current segment (two buffer sets).
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "hydro.h"
#include "hydro_adjoint_math.cuh"
#include "hydro_check.cuh"
#include "hydro_internal.h"
#include "hydro_math.cuh"

namespace hydro {

namespace {

// Tile geometry of the reverse sweeps: SEG cells per line along the sweep axis,
// LANES lines, 8 staged cells of halo on each side and SEG + 8 interfaces per
// line.  FP64 tiles are bound by the FP64 pipe: long lines recompute fewer halo
// interfaces (136 per 128 cells), 256 threads, two blocks per SM at ~120
// registers.  FP32-flux (mixed) tiles are 64 x 4 with one thread per interface
// (288), so that each component's reverse WENO pass is a single round.
template <int PREC>
struct AdjTile {
  static constexpr int SEG = PREC == HYDRO_MIXED ? 64 : 128;
  static constexpr int LANES = PREC == HYDRO_MIXED ? 4 : 2;
  static constexpr int W = SEG + 16;       // staged positions per line: a0-8 .. a0+SEG+7
  static constexpr int NCS = LANES * W;
  static constexpr int NI = SEG + 8;       // interfaces i = a0-4 .. a0+SEG+3
  static constexpr int NIF = LANES * NI;
  static constexpr int NC = LANES * SEG;
  static constexpr int THREADS = PREC == HYDRO_MIXED ? NIF : 256;
};
template <int PREC> __host__ __device__ constexpr int adj_threads() { return AdjTile<PREC>::THREADS; }

template <int PREC, class P>
constexpr size_t adj_smem() {
  using T = AdjTile<PREC>;
  constexpr size_t shadow_words = PREC == HYDRO_MIXED ? 2 * T::NCS : 0;
  return sizeof(P) * (size_t)(16 * T::NCS + 16 * T::NIF + 2 * T::NIF + 15 * T::NC + shadow_words) +
         sizeof(unsigned) * T::NIF;
}

// Flux arithmetic of the adjoint sweeps: the forward's (FP64, or FP32 for mixed).
template <int PREC> struct AdjTypes { using P = double; using Math = MathD; };
template <> struct AdjTypes<HYDRO_MIXED> { using P = float; using Math = MathF; };

struct VjpArgs {
  const double* U;      // FP64: stage state the right-hand side was evaluated on
  const double* lam;    // adjoint of the stage result; a = ascale * lam is the adjoint of L (FP64)
  const float* sh;      // mixed: the forward's FP32 shadow of the stage state, [6][n] = E, M^x, M^y, M^z,
                        // R, om (E one ulp below the FP32 floor where the FP64 recovery floors it)
  const float* lamf;    // mixed: a = ascale * lam, already scaled, in FP32
  void* r;              // output J_L^T a in the flux type (x sweep writes, y and z add)
  double* kbar;         // [2 kMaxJets]: dJ/dk_rad, dJ/dk_coll per jet (one writer per jet and stage)
  double ascale;
  int nx, ny, nz;
  double inv_dx, e_floor, eps_s;
  float inv_dx_f, eps_s_f, e_floor_f;   // the same rounded to FP32 on the host (mixed)
  double rad_per_k, coll_per_k, k_rad, k_coll, t4coef, inv_vol;
  DevDiag* diag;        // status word (and, in the bounds-checked build, the failed check)
  JetStage jets;
};

__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

__device__ __forceinline__ long long bits_of(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ int bits_of(float x) { return __float_as_int(x); }
template <class P> __device__ __forceinline__ P from_bits(long long b) { return __longlong_as_double(b); }
template <> __device__ __forceinline__ float from_bits<float>(long long b) { return __int_as_float((int)b); }

// Moves the adjoints of the ghost slots of one interface to its edge-cell slots:
// slots t < t0 (left of position 0) join slot t0, slots t > t1 (right of position
// n - 1) join slot t1.  Compile-time slot indices, so the arrays stay in registers.
template <class P>
__device__ __forceinline__ void fold_ghost_slots(P (&vf)[8], P (&vu)[8], int t0, int t1) {
  P lf = P(0), lu = P(0), rf = P(0), ru = P(0);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (t < t0) {
      lf += vf[t];
      lu += vu[t];
      vf[t] = P(0);
      vu[t] = P(0);
    }
    if (t > t1) {
      rf += vf[t];
      ru += vu[t];
      vf[t] = P(0);
      vu[t] = P(0);
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (t == t0) {
      vf[t] += lf;
      vu[t] += lu;
    }
    if (t == t1) {
      vf[t] += rf;
      vu[t] += ru;
    }
  }
}

template <int PREC, int DIR>
__global__ void __launch_bounds__(adj_threads<PREC>()) vjp_kernel(const VjpArgs p) {
  constexpr int kAdjThreads = adj_threads<PREC>();
  using P = typename AdjTypes<PREC>::P;
  using Math = typename AdjTypes<PREC>::Math;
  constexpr bool MIXED = PREC == HYDRO_MIXED;
  using T = AdjTile<PREC>;
  constexpr int SEG = T::SEG, LANES = T::LANES, W = T::W, NCS = T::NCS, NI = T::NI, NIF = T::NIF, NC = T::NC;
  constexpr bool FINAL = DIR == 2;
  // cells whose alpha lies within this relative distance of the maximum share its derivative
  constexpr P kTie = MIXED ? P(1e-6) : P(1e-12);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  P* sU = reinterpret_cast<P*>(smem_raw);   // [5][NCS]
  P* sF = sU + 5 * NCS;                     // [5][NCS] F_d/2
  P* sA = sF + 5 * NCS;                     // [5][NCS] adjoint of L (0 outside the grid)
  P* sR = sA + 5 * NCS;                     // [NCS] rho_d
  P* cF = sR + NCS;                         // [8][NIF] adjoint of F_d/2 per stencil slot
  P* cU = cF + 8 * NIF;                     // [8][NIF] direct adjoint of U per stencil slot
  P* sAl = cU + 8 * NIF;                    // [NIF] alpha
  P* sAhb = sAl + NIF;                      // [NIF] adjoint of alpha/2
  P* sFb = sAhb + NIF;                      // [5][NC] gathered adjoint of F_d/2
  P* sUb = sFb + 5 * NC;                    // [5][NC] gathered direct adjoint of U
  P* sRp = sUb + 5 * NC;                    // [5][NC] y, z: r of the cells before this sweep adds to it
  P* sEf = sRp + 5 * NC;                    // mixed: [NCS] signed floored E of the recovery
  P* sOm = sEf + (MIXED ? NCS : 0);         // mixed: [NCS] om = 1 - |M|/E
  unsigned* sTie = reinterpret_cast<unsigned*>(sOm + (MIXED ? NCS : 0));   // [NIF] slots attaining max rho
  P* r_out = static_cast<P*>(p.r);

  const int nx = p.nx, ny = p.ny, nz = p.nz;
  // 32-bit element indices: hydro_adjoint_create admits at most 4e8 cells (7 shadow fields < 2^32)
  const unsigned N = (unsigned)nx * ny * nz;
  const int n_along = DIR == 0 ? nx : (DIR == 1 ? ny : nz);
  const int n_lane = DIR == 0 ? ny : nx;
  int a0, l0;
  if (DIR == 0) { a0 = blockIdx.x * SEG; l0 = blockIdx.y * LANES; }
  else { l0 = blockIdx.x * LANES; a0 = blockIdx.y * SEG; }
  const int fixed = blockIdx.z;
  auto offset = [&](int along, int lane) -> unsigned {
    if (DIR == 0) return ((unsigned)fixed * ny + lane) * nx + along;
    if (DIR == 1) return ((unsigned)fixed * ny + along) * nx + lane;
    return ((unsigned)along * ny + fixed) * nx + lane;
  };
  auto sidx = [&](int lane, int s) { return DIR == 0 ? lane * W + s : s * LANES + lane; };
  auto iidx = [&](int lane, int ii) { return DIR == 0 ? lane * NI + ii : ii * LANES + lane; };
  auto cidx = [&](int lane, int j) { return DIR == 0 ? lane * SEG + j : j * LANES + lane; };

  // ---- adjoint a of L at positions a0-8 .. a0+SEG+7 (zero outside the grid).  A tile
  // whose window holds no nonzero adjoint contributes exactly zero (every term of
  // J_L^T a carries a factor of a): it writes its zeros (x sweep) and stops.  The
  // adjoint of a localised observable starts on a small support that each stage
  // widens by the stencil reach.
  // The charge density R feeds no other field, so its adjoint is zero for an
  // observable of E and M: a block whose R window is exactly zero skips the R
  // pass, which would only add zeros (s_liveR is cleared before the first barrier
  // and set after it).
  __shared__ int s_liveR;
  if (threadIdx.x == 0) s_liveR = 0;
  // Every load of the window (the adjoint, the state and, for y and z, the r values
  // this sweep adds to) is issued before any of them is used, so that the block
  // waits for one round of memory latency.
  constexpr int RND = (NCS + kAdjThreads - 1) / kAdjThreads;   // positions per thread
  constexpr int NSH = MIXED ? 6 : 5;                            // state words per position
  constexpr bool RPRE = DIR != 0;
  P av[RND][5], uv[RND][NSH], rv[RND][5];
  bool live = false, liveR = false;
#pragma unroll
  for (int rd = 0; rd < RND; ++rd) {
    const int c = threadIdx.x + rd * kAdjThreads;
    if (c < NCS) {
      int lane, s;
      if (DIR == 0) { lane = c / W; s = c - lane * W; }
      else { s = c / LANES; lane = c - s * LANES; }
      const int ga = a0 - 8 + s;
      const int gl = l0 + lane;
      const bool inside = ga >= 0 && ga < n_along && gl < n_lane;
      const unsigned oa = HYDRO_CELL_AT(offset(inside ? ga : 0, gl < n_lane ? gl : 0), N, kSiteAdjWindow, 0, p.diag);
      const unsigned o =
          HYDRO_CELL_AT(offset(clampi(ga, n_along), gl < n_lane ? gl : n_lane - 1), N, kSiteAdjWindow, 0, p.diag);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        if constexpr (MIXED) av[rd][q] = inside ? p.lamf[q * N + oa] : P(0);
        else av[rd][q] = inside ? p.ascale * p.lam[q * N + oa] : P(0);
      }
#pragma unroll
      for (int f = 0; f < NSH; ++f) {
        if constexpr (MIXED) uv[rd][f] = p.sh[f * N + o];
        else uv[rd][f] = p.U[f * N + o];
      }
      if constexpr (RPRE) {
        const bool cell = inside && s >= 8 && s < 8 + SEG;
#pragma unroll
        for (int k = 0; k < 5; ++k) rv[rd][k] = cell ? r_out[k * N + oa] : P(0);
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        sA[q * NCS + c] = av[rd][q];
        live |= av[rd][q] != P(0);
        if (q == 4) liveR |= av[rd][q] != P(0);
      }
    }
  }
  if (!__syncthreads_or(live)) {
    if (DIR == 0) {
      for (int c = threadIdx.x; c < NC; c += kAdjThreads) {
        int lane, j;
        lane = c / SEG;
        j = c - lane * SEG;
        if (a0 + j >= n_along || l0 + lane >= n_lane) continue;
        const unsigned o = HYDRO_CELL_AT(offset(a0 + j, l0 + lane), N, kSiteAdjResult, 0, p.diag);
        for (int k = 0; k < 5; ++k) r_out[k * N + o] = P(0);
      }
    }
    return;
  }
  if (liveR) s_liveR = 1;

  // ---- U, F_d/2, rho_d at positions a0-8 .. a0+SEG+7 (clamped), from the loaded window
#pragma unroll
  for (int rd = 0; rd < RND; ++rd) {
    const int c = threadIdx.x + rd * kAdjThreads;
    if (c < NCS) {
      int lane, s;
      if (DIR == 0) { lane = c / W; s = c - lane * W; }
      else { s = c / LANES; lane = c - s * LANES; }
      P e, vx, vy, vz;
      const P E = uv[rd][0], Mx = uv[rd][1], My = uv[rd][2], Mz = uv[rd][3], R = uv[rd][4];
      int hit = 0;
      if constexpr (MIXED) {
        // the recovery of the forward's shadow (cons_to_prim_shadow): the floor acts
        // where the shadow's E lies below the FP32 floor
        const float Efs = E >= p.e_floor_f ? E : -p.e_floor_f;
        cons_to_prim_om(Efs, Mx, My, Mz, uv[rd][5], e, vx, vy, vz, hit);
        sEf[c] = Efs;
        sOm[c] = uv[rd][5];
      } else {
        cons_to_prim<MathD>(E, Mx, My, Mz, p.e_floor, e, vx, vy, vz, hit);
      }
      const P pr = e * P(1.0 / 3.0);
      const P vd = DIR == 0 ? vx : (DIR == 1 ? vy : vz);
      sU[c] = E; sU[NCS + c] = Mx; sU[2 * NCS + c] = My; sU[3 * NCS + c] = Mz; sU[4 * NCS + c] = R;
      sF[c] = P(0.5) * (DIR == 0 ? Mx : (DIR == 1 ? My : Mz));
      sF[NCS + c] = P(0.5) * (Mx * vd + (DIR == 0 ? pr : P(0)));
      sF[2 * NCS + c] = P(0.5) * (My * vd + (DIR == 1 ? pr : P(0)));
      sF[3 * NCS + c] = P(0.5) * (Mz * vd + (DIR == 2 ? pr : P(0)));
      sF[4 * NCS + c] = P(0.5) * (R * vd);
      sR[c] = spectral_radius<Math>(vd, vx * vx + vy * vy + vz * vz);
      if constexpr (RPRE) {
        if (s >= 8 && s < 8 + SEG) {
#pragma unroll
          for (int k = 0; k < 5; ++k) sRp[k * NC + cidx(lane, s - 8)] = rv[rd][k];
        }
      }
    }
  }
  __syncthreads();

  // ---- alpha and the slots that attain it, per interface i = a0-4+ii (valid for -1 <= i <= n-1)
  for (int it = threadIdx.x; it < NIF; it += kAdjThreads) {
    int lane, ii;
    if (DIR == 0) { lane = it / NI; ii = it - lane * NI; }
    else { ii = it / LANES; lane = it - ii * LANES; }
    const int i = a0 - 4 + ii;
    const bool valid = i >= -1 && i <= n_along - 1 && l0 + lane < n_lane;
    // rho >= 0: compared as bit patterns (integer pipe), which order like the values
    using I = typename std::conditional<sizeof(P) == 8, long long, int>::type;
    I alb = 0;
    for (int t = 0; t < 8; ++t) {
      const I rb = bits_of(sR[sidx(lane, ii + 1 + t)]);
      alb = rb > alb ? rb : alb;
    }
    const P al = from_bits<P>(alb);
    unsigned mask = 0;
    if (valid) {
      const I thr = bits_of(al * (P(1) - kTie));
      for (int t = 0; t < 8; ++t)
        if (bits_of(sR[sidx(lane, ii + 1 + t)]) >= thr) mask |= 1u << t;
    }
    sAl[iidx(lane, ii)] = al;
    sTie[iidx(lane, ii)] = mask;
    sAhb[iidx(lane, ii)] = P(0);
  }
  __syncthreads();
  const int nq = s_liveR ? 5 : 4;   // block-uniform

  // ---- per component: reverse WENO at every interface, then gather per cell
  for (int q = 0; q < nq; ++q) {
    for (int it = threadIdx.x; it < NIF; it += kAdjThreads) {
      int lane, ii;
      if (DIR == 0) { lane = it / NI; ii = it - lane * NI; }
      else { ii = it / LANES; lane = it - ii * LANES; }
      const int x = iidx(lane, ii);
      P* cf = cF + x;   // slot t at cf[t * NIF]: consecutive interfaces hit consecutive banks
      P* cu = cU + x;
      // adjoint of Fhat_{i+1/2}: L_i holds -Fhat inv_dx, L_{i+1} holds +Fhat inv_dx; the
      // reverse of an interface whose flux adjoint is zero is zero
      const P g = (sA[q * NCS + sidx(lane, ii + 5)] - sA[q * NCS + sidx(lane, ii + 4)]) *
                  (MIXED ? (P)p.inv_dx_f : (P)p.inv_dx);
      if (sTie[x] == 0u || g == P(0)) {
#pragma unroll
        for (int t = 0; t < 8; ++t) { cf[t * NIF] = P(0); cu[t * NIF] = P(0); }
        continue;
      }
      const P ah = P(0.5) * sAl[x];
      P u[8], fh[8];
      for (int t = 0; t < 8; ++t) {
        u[t] = sU[q * NCS + sidx(lane, ii + 1 + t)];
        fh[t] = sF[q * NCS + sidx(lane, ii + 1 + t)];
      }
      P gp[7], gm[7];
      if constexpr (MIXED) {
        // f+ and the mirrored f- (cells i+4 .. i-2) in the two lanes of packed FP32x2,
        // split by scalar FMAs that write the lanes directly
        float2 fpm[7], gb[7];
#pragma unroll
        for (int t = 0; t < 7; ++t) fpm[t] = make_float2(fmaf(ah, u[t], fh[t]), fmaf(-ah, u[7 - t], fh[7 - t]));
        weno7_vjp_pair(fpm, p.eps_s_f, make_float2(g, g), gb);
#pragma unroll
        for (int t = 0; t < 7; ++t) {
          gp[t] = gb[t].x;
          gm[t] = gb[t].y;
        }
      } else {
        P fp[7], fm[7];
        for (int t = 0; t < 7; ++t) {
          fp[t] = fh[t] + ah * u[t];
          fm[t] = fh[7 - t] - ah * u[7 - t];   // mirrored: cells i+4 .. i-2
        }
        weno7_vjp<P>(fp, (P)p.eps_s, g, gp);
        weno7_vjp<P>(fm, (P)p.eps_s, g, gm);
      }
      P ahb = P(0), vf[8], vu[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const P bp = t <= 6 ? gp[t] : P(0);
        const P bm = t >= 1 ? gm[7 - t] : P(0);
        vf[t] = bp + bm;
        vu[t] = ah * (bp - bm);
        ahb += u[t] * (bp - bm);
      }
      // slot t is position i - 3 + t; a position outside the grid is a clamped copy
      // of the edge cell, whose adjoint it therefore joins
      const int i = a0 - 4 + ii;
      if (i < 3 || i > n_along - 5) fold_ghost_slots(vf, vu, 3 - i, n_along + 2 - i);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        cf[t * NIF] = vf[t];
        cu[t * NIF] = vu[t];
      }
      sAhb[x] += ahb;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NC; c += kAdjThreads) {
      int lane, j;
      if (DIR == 0) { lane = c / SEG; j = c - lane * SEG; }
      else { j = c / LANES; lane = c - j * LANES; }
      P fb = P(0), ub = P(0);
      // cell j is slot 7 - k of interface j + k (the ghost slots are folded into the
      // edge cells' slots; interfaces outside the grid hold zeros)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int x = iidx(lane, j + k);
        fb += cF[(7 - k) * NIF + x];
        ub += cU[(7 - k) * NIF + x];
      }
      sFb[q * NC + cidx(lane, j)] = fb;
      sUb[q * NC + cidx(lane, j)] = ub;
    }
    __syncthreads();
  }

  // ---- per cell: adjoint of rho from the interfaces whose max it attains, then the chain rule
  for (int c = threadIdx.x; c < NC; c += kAdjThreads) {
    int lane, j;
    if (DIR == 0) { lane = c / SEG; j = c - lane * SEG; }
    else { j = c / LANES; lane = c - j * LANES; }
    const int gcell = a0 + j, gl = l0 + lane;
    if (gcell >= n_along || gl >= n_lane) continue;
    // cell gcell is slot 7 - k of interface j + k (the edge cells also own the
    // clamped ghost slots beyond them); each tying slot gets an equal share
    P rhob = P(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int x = iidx(lane, j + k);
      const unsigned mask = sTie[x];
      unsigned own = (mask >> (7 - k)) & 1u;
      if (gcell == 0) own += __popc(mask & ((1u << (7 - k)) - 1u));
      if (gcell == n_along - 1) own += __popc(mask >> (8 - k));
      // the equal share: one reciprocal of the tie count (1..8; exact for 1, 2, 4, 8)
      if (own) rhob += P(0.5) * (P)own * sAhb[x] * Math::rcp((P)__popc(mask));
    }
    const int sc = sidx(lane, j + 8);
    const unsigned o = HYDRO_CELL_AT(offset(gcell, gl), N, kSiteAdjResult, 0, p.diag);
    const P Mx = sU[NCS + sc], My = sU[2 * NCS + sc], Mz = sU[3 * NCS + sc], R = sU[4 * NCS + sc];
    P e, vx, vy, vz;
    C2PTape<P> tape;
    if constexpr (MIXED) cons_to_prim_om_tape(sEf[sc], Mx, My, Mz, sOm[sc], tape, e, vx, vy, vz);
    else cons_to_prim_tape(sU[sc], Mx, My, Mz, p.e_floor, tape, e, vx, vy, vz);
    const P v[3] = {vx, vy, vz};
    const P vd = v[DIR];
    const int ci = cidx(lane, j);
    // F/2 adjoint -> F adjoint
    P Fb[5];
    for (int k = 0; k < 5; ++k) Fb[k] = k < nq ? P(0.5) * sFb[k * NC + ci] : P(0);
    P Mb[3] = {P(0), P(0), P(0)}, vb[3] = {P(0), P(0), P(0)}, Rb = P(0), pb = P(0);
    const P M[3] = {Mx, My, Mz};
    Mb[DIR] += Fb[0];
    for (int k = 0; k < 3; ++k) {
      Mb[k] += Fb[1 + k] * vd;
      vb[DIR] += Fb[1 + k] * M[k];
    }
    pb += Fb[1 + DIR];
    Rb += Fb[4] * vd;
    vb[DIR] += Fb[4] * R;
    P d_vd, d_v2;
    spectral_radius_grad<Math>(vd, vx * vx + vy * vy + vz * vz, d_vd, d_v2);
    vb[DIR] += rhob * d_vd;
    for (int k = 0; k < 3; ++k) vb[k] += rhob * d_v2 * P(2) * v[k];
    P Eb = sUb[ci];
    P Mbx = sUb[NC + ci] + Mb[0], Mby = sUb[2 * NC + ci] + Mb[1], Mbz = sUb[3 * NC + ci] + Mb[2];
    if (nq == 5) Rb += sUb[4 * NC + ci];
    c2p_vjp_core<Math>(tape.m, tape.s, tape.r, tape.v, tape.vs, tape.invE, tape.nx, tape.ny, tape.nz, tape.capped,
                       tape.floored, pb * P(1.0 / 3.0), vb[0], vb[1], vb[2], Eb, Mbx, Mby, Mbz);
    const P out[5] = {Eb, Mbx, Mby, Mbz, Rb};
    if (DIR == 0) {
      for (int k = 0; k < 5; ++k) r_out[k * N + o] = out[k];
    } else {
      for (int k = 0; k < 5; ++k) r_out[k * N + o] = sRp[k * NC + ci] + out[k];
    }
  }

  // ---- z sweep: adjoint of the jet source (Eqs. 2-3) at the jet cells of this
  // tile, one thread, after the cells' own contributions (global writes of the
  // block are visible to it after the barrier)
  if constexpr (FINAL) {
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int jn = 0; jn < p.jets.n; ++jn) {
        const int* cl = p.jets.cell[jn];
        if (cl[0] < 0 || cl[1] != fixed || cl[2] < a0 || cl[2] >= a0 + SEG || cl[2] >= n_along || cl[0] < l0 ||
            cl[0] >= l0 + LANES)
          continue;
        const int j = cl[2] - a0, lane = cl[0] - l0;
        const int sc = sidx(lane, j + 8);
        const unsigned o = HYDRO_CELL_AT(offset(cl[2], cl[0]), N, kSiteAdjJet, 0, p.diag);
        // S0 = inv_vol (k_rad C T^3 l / hc^2 + k_coll C T^2 / hc), T = (e t4)^(1/4): S = (S0, n S0, 0).
        // T comes from the recovery the forward used at the jet cell: FP64 from the
        // FP64 state, or (mixed) FP32 from the shadow; its derivative in FP64.
        double Ed, Mxd, Myd, Mzd, es;
        if constexpr (MIXED) {
          const float* S = p.sh;
          float ef, vxf, vyf, vzf, v2f, rdf;
          int hs = 0;
          cons_to_prim_shadow_rho(S[o], S[N + o], S[2 * N + o], S[3 * N + o], S[5 * N + o], p.e_floor_f, ef, vxf,
                                  vyf, vzf, v2f, rdf, hs);
          Ed = S[o]; Mxd = S[N + o]; Myd = S[2 * N + o]; Mzd = S[3 * N + o];
          es = ef;
        } else {
          Ed = p.U[o]; Mxd = p.U[N + o]; Myd = p.U[2 * N + o]; Mzd = p.U[3 * N + o];
          double vsx, vsy, vsz;
          int hs = 0;
          cons_to_prim<MathD>(Ed, Mxd, Myd, Mzd, p.e_floor, es, vsx, vsy, vsz, hs);
        }
        const double aE = sA[sc], aMx = sA[NCS + sc], aMy = sA[2 * NCS + sc], aMz = sA[3 * NCS + sc];
        const double Sb = aE + p.jets.dir[jn][0] * aMx + p.jets.dir[jn][1] * aMy + p.jets.dir[jn][2] * aMz;
        const double T = temperature(es, p.t4coef);
        const double l = p.jets.ell[jn];
        p.kbar[2 * jn] += Sb * p.rad_per_k * T * T * T * l * p.inv_vol;
        p.kbar[2 * jn + 1] += Sb * p.coll_per_k * T * T * p.inv_vol;
        if (es > 0.0 && T > 0.0) {
          const double dS_dT = (3.0 * p.k_rad * p.rad_per_k * T * T * l + 2.0 * p.k_coll * p.coll_per_k * T) * p.inv_vol;
          const double dT_de = T / (4.0 * es);
          double sE = 0.0, sMx = 0.0, sMy = 0.0, sMz = 0.0;
          cons_to_prim_vjp(Ed, Mxd, Myd, Mzd, p.e_floor, Sb * dS_dT * dT_de, 0.0, 0.0, 0.0, sE, sMx, sMy, sMz);
          r_out[o] += (P)sE;
          r_out[N + o] += (P)sMx;
          r_out[2 * N + o] += (P)sMy;
          r_out[3 * N + o] += (P)sMz;
        }
      }
    }
  }
}

template <int PREC, int DIR>
cudaError_t launch_vjp(const VjpArgs& p, cudaStream_t s) {
  using P = typename AdjTypes<PREC>::P;
  constexpr size_t smem = adj_smem<PREC, P>();
  constexpr int SEG = AdjTile<PREC>::SEG, LANES = AdjTile<PREC>::LANES;
  dim3 grid;
  if (DIR == 0) grid = dim3((p.nx + SEG - 1) / SEG, (p.ny + LANES - 1) / LANES, p.nz);
  else if (DIR == 1) grid = dim3((p.nx + LANES - 1) / LANES, (p.ny + SEG - 1) / SEG, p.nz);
  else grid = dim3((p.nx + LANES - 1) / LANES, (p.nz + SEG - 1) / SEG, p.ny);
  auto kern = vjp_kernel<PREC, DIR>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<grid, adj_threads<PREC>(), smem, s>>>(p);
  return cudaGetLastError();
}

// Reverse of one stage combination Uout = ca U0 + cb (Uk + dt L(Uk)), in FP64;
// r is the adjoint of the right-hand side in the flux type.
// mode 0 (stage 3): lamB = cb lamA + r;  lam0 = ca lamA
// mode 1 (stage 2): lamA = cb lamB + r;  lam0 += ca lamB
// mode 2 (stage 1): lam0 += lamA + r
// Mixed precision: the adjoint the next reverse sweep reads (lamB, lamA, lam0
// for modes 0, 1, 2) also goes to lamf, scaled by that sweep's fscale, in FP32.
template <class R>
__global__ void adj_combine_kernel(int mode, double ca, double cb, double* lamA, double* lamB, double* lam0,
                                   const R* r, size_t n, float* lamf, float fscale) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    // FP32 <-> FP64 conversions on the integer pipe (B300 runs FP64 at 1/64 rate)
    double ri;
    if constexpr (sizeof(R) == 4) ri = f2d(r[i]);
    else ri = r[i];
    double next;
    if (mode == 0) {
      const double la = lamA[i];
      next = cb * la + ri;
      lamB[i] = next;
      lam0[i] = ca * la;
    } else if (mode == 1) {
      const double lb = lamB[i];
      next = cb * lb + ri;
      lamA[i] = next;
      lam0[i] += ca * lb;
    } else {
      next = lam0[i] + (lamA[i] + ri);
      lam0[i] = next;
    }
    if (lamf) lamf[i] = fscale * d2f_rn(next);
  }
}

__global__ void scale_to_float_kernel(const double* x, float* y, double scale, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = d2f_rn(scale * x[i]);
}

struct ConeArgs {
  double apex[3], axis[3], cos_half, rmax2, dx, vol;
  int nx, ny, nz;
};

__device__ __forceinline__ bool in_cone(const ConeArgs& c, int i, int j, int k) {
  const double x = (i + 0.5 - 0.5 * c.nx) * c.dx - c.apex[0];
  const double y = (j + 0.5 - 0.5 * c.ny) * c.dx - c.apex[1];
  const double z = (k + 0.5 - 0.5 * c.nz) * c.dx - c.apex[2];
  const double r2 = x * x + y * y + z * z;
  if (!(r2 < c.rmax2)) return false;
  return x * c.axis[0] + y * c.axis[1] + z * c.axis[2] >= c.cos_half * sqrt(r2);
}

// Partial sums of E dx^3 over the cone, one per block (summed on the host in order).
__global__ void cone_energy_kernel(const double* U, ConeArgs c, double* partial) {
  __shared__ double red[256];
  const size_t n = (size_t)c.nx * c.ny * c.nz;
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % c.nx), iy = (int)((i / c.nx) % c.ny), iz = (int)(i / ((size_t)c.nx * c.ny));
    if (in_cone(c, ix, iy, iz)) acc += U[i] * c.vol;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Seed of the reverse sweep: dJ/dU = g dx^3 on E inside the cone.
__global__ void cone_seed_kernel(double* lam, ConeArgs c, double g) {
  const size_t n = (size_t)c.nx * c.ny * c.nz;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % c.nx), iy = (int)((i / c.nx) % c.ny), iz = (int)(i / ((size_t)c.nx * c.ny));
    lam[i] = in_cone(c, ix, iy, iz) ? g * c.vol : 0.0;
    for (int q = 1; q < 5; ++q) lam[q * n + i] = 0.0;
  }
}

// dJ/de of the initial state at fixed u^i and n: E = (4/3) e gamma^2 - e/3,
// M^i = (4/3) e gamma u^i, R = n gamma.
__global__ void grad_e_kernel(const double* prim, const double* lam, double* grad, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double ux = prim[n + i], uy = prim[2 * n + i], uz = prim[3 * n + i];
    const double g2 = 1.0 + (ux * ux + uy * uy + uz * uz);
    const double g = sqrt(g2);
    grad[i] = lam[i] * (4.0 / 3.0 * g2 - 1.0 / 3.0) +
              (4.0 / 3.0) * g * (lam[n + i] * ux + lam[2 * n + i] * uy + lam[3 * n + i] * uz);
  }
}

unsigned grid_1d(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b < 148 * 16 ? (b > 0 ? b : 1) : 148 * 16);
}

}  // namespace
}  // namespace hydro

using namespace hydro;

// One set of segment buffers: the step and stage states of up to `every` steps
// recomputed from a checkpoint.  FP64 keeps the stage states in FP64 (U1, U2 of
// each step); mixed precision keeps what its reverse sweeps read, the FP32
// shadows of the three stage states of each step (the stage states themselves
// are FP32 increments in the accumulator while the step runs).
struct AdjSet {
  std::vector<double*> seg;     // every + 1 step states
  std::vector<double*> stages;  // FP64: 2 every stage states
  std::vector<float*> shd;      // mixed: 3 every + 1 shadows [6][n] (the last one: of the segment's end state)
  double* rhs = nullptr;        // accumulator of the sweeps
  double* prim = nullptr;       // FP64: primitive cache of the x sweep
};

struct hydro_adjoint {
  hydro_config cfg;
  size_t n = 0;
  int nsteps = 0, every = 0, nckpt = 0;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  bool owns_ws = false;          // ws came from cudaMalloc (no caller workspace)
  std::vector<double*> ckpt;     // states at steps 0, every, 2 every, ...
  // two segment buffer sets: the set of segment k is (nckpt - 1 - k) & 1; one is
  // refilled on a side stream while the main stream reverses the other
  AdjSet set[2];
  cudaStream_t side = nullptr;
  cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr}, ev_start = nullptr;
  double *lamA = nullptr, *lamB = nullptr, *lam0 = nullptr;   // adjoint states (roles rotate per step)
  double* r = nullptr;           // J_L^T a of the stage under reverse, in the flux type
  double* prim = nullptr;        // the forward's initial primitives (for dJ/de)
  float* lamf = nullptr;         // mixed: FP32 scaled adjoint input of the next reverse sweep [5][n]
  double* kbar = nullptr;        // [2]
  double* partial = nullptr;     // cone partial sums
  DevDiag* diag = nullptr;
  int njet = 0;
  double jx0[kMaxJets][3], jn[kMaxJets][3], jt[kMaxJets];
  ConeArgs cone;
  bool forward_done = false;
  bool last_kept = false;        // the forward left the last segment's states in set 0
  double J = 0.0;
};

namespace {

constexpr unsigned kConeBlocks = 512;

void jet_stage(const hydro_adjoint* a, double t, JetStage& js) {
  std::memset(&js, 0, sizeof(js));
  const int N[3] = {a->cfg.nx, a->cfg.ny, a->cfg.nz};
  js.n = a->njet;
  for (int j = 0; j < a->njet; ++j) {
    jet_cell_at(a->jx0[j], a->jn[j], a->jt[j], t, a->cfg.dx, N, js.cell[j], &js.ell[j]);
    for (int ax = 0; ax < 3; ++ax) js.dir[j][ax] = a->jn[j][ax];
  }
}

SweepArgs sweep_base(const hydro_adjoint* a) {
  SweepArgs s;
  std::memset(&s, 0, sizeof(s));
  const hydro_config& g = a->cfg;
  s.diag = a->diag;
  grid_args_from_config(g, s);   // (outflow, no test hooks: the adjoint accepts no other)
  return s;
}

// One forward step from `in` (step index n, position i in its segment set) to
// `out`, as hydro_step runs it (same kernels, tensor maps where the grid admits
// them): FP64 writes the stage states to the set's stages[2i], stages[2i + 1];
// mixed precision reads the shadow of `in` from shd[3i] (computed here at i = 0)
// and writes the shadows of the next stage states and of `out` to shd[3i + 1 ..
// 3i + 3].
cudaError_t forward_step(hydro_adjoint* a, int64_t n, AdjSet& S, int i, const double* in, double* out,
                         cudaStream_t stream) {
  const hydro_config& g = a->cfg;
  const bool mixed = g.precision == HYDRO_MIXED;
  SweepArgs s = sweep_base(a);
  s.rhs = S.rhs;
  s.U0 = in;
  s.P = mixed ? nullptr : S.prim;
  const double vol = g.dx * g.dx * g.dx;
  cudaError_t err = cudaSuccess;
  SweepMaps maps[3][3];
  bool tma;
  if (mixed) {
    if (i == 0) err = launch_shadow(in, S.shd[0], a->n, g.e_floor, stream);
    void* bufs[3] = {const_cast<double*>(in), const_cast<double*>(in), const_cast<double*>(in)};
    void* shs[3] = {S.shd[3 * i], S.shd[3 * i + 1], S.shd[3 * i + 2]};
    tma = encode_sweep_tmaps(g.precision, 7, bufs, S.rhs, g.nx, g.ny, g.nz, maps, shs);
  } else {
    void* bufs[3] = {const_cast<double*>(in), S.stages[2 * i], S.stages[2 * i + 1]};
    tma = encode_sweep_tmaps(g.precision, 7, bufs, S.rhs, g.nx, g.ny, g.nz, maps);
  }
  for (int st = 0; st < 3 && err == cudaSuccess; ++st) {
    jet_stage(a, g.t0 + ((double)n + kRK3C[st]) * g.dt, s.jets);
    s.src.wdt_vol = g.dt * kRK3W[st] * vol;
    if (mixed) {   // stage states as FP32 increments over U0 in the accumulator
      s.U = in;
      s.Uout = st == 2 ? out : nullptr;
      s.S = S.shd[3 * i + st];
      s.Sout = S.shd[3 * i + st + 1];
    } else {
      s.U = st == 0 ? in : S.stages[2 * i + st - 1];
      s.Uout = st == 2 ? out : S.stages[2 * i + st];
    }
    s.a = kRK3A[st];
    s.b = kRK3B[st];
    for (int d = 0; d < 3 && err == cudaSuccess; ++d)
      err = launch_sweep(g.precision, 7, d, s, stream, tma ? &maps[st][d] : nullptr);
  }
  return err;
}

// The reverse sweeps of stage st of step n, on the stage state Uk (FP64) or its
// shadow sh (mixed).
cudaError_t vjp(hydro_adjoint* a, int64_t n, int st, const double* Uk, const float* sh, const double* lam,
                double ascale) {
  VjpArgs p;
  std::memset(&p, 0, sizeof(p));
  const hydro_config& g = a->cfg;
  p.U = Uk;
  p.sh = sh;
  p.lam = lam;
  p.r = a->r;
  p.kbar = a->kbar;
  p.diag = a->diag;
  p.ascale = ascale;
  p.nx = g.nx;
  p.ny = g.ny;
  p.nz = g.nz;
  p.inv_dx = 1.0 / g.dx;
  p.e_floor = g.e_floor;
  p.eps_s = kW7EpsScale * g.weno_eps;
  p.inv_dx_f = (float)p.inv_dx;
  p.eps_s_f = (float)p.eps_s;
  p.e_floor_f = (float)g.e_floor;
  p.rad_per_k = g.cr_over_cf / (g.hbarc * g.hbarc);
  p.coll_per_k = g.cr_over_cf / g.hbarc;
  p.k_rad = g.k_rad;
  p.k_coll = g.k_coll;
  const SourceCoef sc = source_coef(g);
  p.t4coef = sc.t4coef;
  p.inv_vol = sc.inv_vol;
  jet_stage(a, g.t0 + ((double)n + kRK3C[st]) * g.dt, p.jets);
  cudaError_t err;
  if (g.precision == HYDRO_MIXED) {
    p.lamf = a->lamf;
    err = launch_vjp<HYDRO_MIXED, 0>(p, a->stream);
    if (err == cudaSuccess) err = launch_vjp<HYDRO_MIXED, 1>(p, a->stream);
    if (err == cudaSuccess) err = launch_vjp<HYDRO_MIXED, 2>(p, a->stream);
  } else {
    err = launch_vjp<HYDRO_FP64, 0>(p, a->stream);
    if (err == cudaSuccess) err = launch_vjp<HYDRO_FP64, 1>(p, a->stream);
    if (err == cudaSuccess) err = launch_vjp<HYDRO_FP64, 2>(p, a->stream);
  }
  return err;
}

// Reverse of the stage combination of stage st; the reverse sweep that follows
// is stage st - 1 of the same step, or stage 3 of the previous step.
// The charge density R is passive (it feeds no other field) and the cone energy
// does not depend on it, so its adjoint stays exactly zero: the stage
// combinations carry the four fields E, M^x, M^y, M^z, and the R fields of the
// adjoint arrays are zeroed once per backward.
constexpr int kAdjFields = 4;

cudaError_t combine(hydro_adjoint* a, int mode, int st) {
  const size_t nf = kAdjFields * a->n;
  const double fscale = kRK3B[st == 0 ? 2 : st - 1] * a->cfg.dt;
  if (a->cfg.precision == HYDRO_MIXED)
    adj_combine_kernel<float><<<grid_1d(nf), 256, 0, a->stream>>>(
        mode, kRK3A[st], kRK3B[st], a->lamA, a->lamB, a->lam0, reinterpret_cast<const float*>(a->r), nf, a->lamf,
        (float)fscale);
  else
    adj_combine_kernel<double><<<grid_1d(nf), 256, 0, a->stream>>>(
        mode, kRK3A[st], kRK3B[st], a->lamA, a->lamB, a->lam0, a->r, nf, nullptr, 0.0f);
  return cudaGetLastError();
}

// The run configurations the adjoint supports: FP64 or mixed, outflow, WENO7,
// the forward's grid limits, at least one step and checkpoint interval.
bool adjoint_config_ok(const hydro_config* cfg, int32_t nsteps, int32_t checkpoint_every) {
  if (!config_valid(cfg, kCheckGrid | kCheckWorkspace)) return false;
  if ((cfg->precision != HYDRO_FP64 && cfg->precision != HYDRO_MIXED) || cfg->boundary != HYDRO_OUTFLOW ||
      cfg->weno_order != 7 || cfg->test_withhold_copies != 0 || cfg->test_check_tighten != 0)
    return false;
  return nsteps >= 1 && checkpoint_every >= 1;
}

// Lays out the run's buffers from base (256-byte aligned pieces) and returns the
// bytes they take; with base == nullptr only the size is computed.
size_t adjoint_layout(hydro_adjoint* a, char* base) {
  char* p = base;
  size_t used = 0;
  auto take = [&](size_t b) {
    char* q = p;
    const size_t s = (b + 255) / 256 * 256;
    used += s;
    if (p) p += s;
    return q;
  };
  const bool mixed = a->cfg.precision == HYDRO_MIXED;
  const size_t n = a->n, f5 = 5 * n * sizeof(double), f6 = 6 * n * sizeof(float);
  a->ckpt.clear();
  for (int k = 0; k < a->nckpt; ++k) a->ckpt.push_back(reinterpret_cast<double*>(take(f5)));
  for (AdjSet& S : a->set) {
    S.seg.clear();
    S.stages.clear();
    S.shd.clear();
    for (int k = 0; k <= a->every; ++k) S.seg.push_back(reinterpret_cast<double*>(take(f5)));
    if (mixed) {
      for (int k = 0; k <= 3 * a->every; ++k) S.shd.push_back(reinterpret_cast<float*>(take(f6)));
    } else {
      for (int k = 0; k < 2 * a->every; ++k) S.stages.push_back(reinterpret_cast<double*>(take(f5)));
      S.prim = reinterpret_cast<double*>(take(f5));
    }
    S.rhs = reinterpret_cast<double*>(take(f5));
  }
  a->lamA = reinterpret_cast<double*>(take(f5));
  a->lamB = reinterpret_cast<double*>(take(f5));
  a->lam0 = reinterpret_cast<double*>(take(f5));
  a->r = reinterpret_cast<double*>(take(f5));
  a->prim = reinterpret_cast<double*>(take(f5));
  if (mixed) a->lamf = reinterpret_cast<float*>(take(5 * n * sizeof(float)));
  a->kbar = reinterpret_cast<double*>(take(2 * kMaxJets * sizeof(double)));
  a->partial = reinterpret_cast<double*>(take(kConeBlocks * sizeof(double)));
  a->diag = reinterpret_cast<DevDiag*>(take(sizeof(DevDiag)));
  return used;
}

// Fills the size fields of a run (grid cells, steps, checkpoint interval and count).
void adjoint_sizes(hydro_adjoint* a, const hydro_config* cfg, int32_t nsteps, int32_t checkpoint_every) {
  a->cfg = *cfg;
  a->n = (size_t)cfg->nx * cfg->ny * cfg->nz;
  a->nsteps = nsteps;
  a->every = checkpoint_every < nsteps ? checkpoint_every : nsteps;
  a->nckpt = (nsteps + a->every - 1) / a->every;
}

}  // namespace

extern "C" {

hydro_status hydro_adjoint_workspace_size(const hydro_config* cfg, int32_t nsteps, int32_t checkpoint_every,
                                          size_t* bytes) {
  if (!bytes || !adjoint_config_ok(cfg, nsteps, checkpoint_every)) return HYDRO_EINVAL;
  hydro_adjoint probe;
  adjoint_sizes(&probe, cfg, nsteps, checkpoint_every);
  *bytes = adjoint_layout(&probe, nullptr);
  return HYDRO_OK;
}

hydro_status hydro_adjoint_create(const hydro_config* cfg, int32_t nsteps, int32_t checkpoint_every,
                                  const double apex[3], const double axis[3], double half_angle_deg, double rmax,
                                  hydro_adjoint** out) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  if (!adjoint_config_ok(cfg, nsteps, checkpoint_every) || !apex || !axis) return HYDRO_EINVAL;
  const double al = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
  if (!(al > 0.0) || !(rmax > 0.0) || !(half_angle_deg > 0.0 && half_angle_deg < 180.0)) return HYDRO_EINVAL;
  hydro_adjoint* a = new (std::nothrow) hydro_adjoint;
  if (!a) return HYDRO_ENOMEM;
  adjoint_sizes(a, cfg, nsteps, checkpoint_every);
  a->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  for (int k = 0; k < 3; ++k) {
    a->cone.apex[k] = apex[k];
    a->cone.axis[k] = axis[k] / al;
  }
  a->cone.cos_half = std::cos(half_angle_deg * M_PI / 180.0);
  a->cone.rmax2 = rmax * rmax;
  a->cone.dx = cfg->dx;
  a->cone.vol = cfg->dx * cfg->dx * cfg->dx;
  a->cone.nx = cfg->nx;
  a->cone.ny = cfg->ny;
  a->cone.nz = cfg->nz;
  // buffers: checkpoints, the segment's step states and stage states, adjoints, scratch
  const size_t bytes = adjoint_layout(a, nullptr);
  if (cfg->workspace) {
    if (cfg->workspace_bytes < bytes) {
      delete a;
      return HYDRO_ENOMEM;
    }
    a->ws = static_cast<char*>(cfg->workspace);
  } else {
    if (cudaMalloc(&a->ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      delete a;
      return HYDRO_ENOMEM;
    }
    a->owns_ws = true;
  }
  adjoint_layout(a, a->ws);
  bool ok = cudaStreamCreateWithFlags(&a->side, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&a->ev_start, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < 2 && ok; ++k)
    ok = cudaEventCreateWithFlags(&a->ev_ready[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&a->ev_free[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    hydro_adjoint_destroy(a);
    return HYDRO_ECUDA;
  }
  *out = a;
  return HYDRO_OK;
}

hydro_status hydro_adjoint_add_jet(hydro_adjoint* a, const double x0[3], const double dir[3], double t_start) {
  if (!a || !x0 || !dir || a->njet >= kMaxJets || !std::isfinite(t_start)) return HYDRO_EINVAL;
  const double len = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (!(len > 0.0) || !std::isfinite(len)) return HYDRO_EINVAL;
  for (int k = 0; k < 3; ++k) {
    a->jx0[a->njet][k] = x0[k];
    a->jn[a->njet][k] = dir[k] / len;
  }
  a->jt[a->njet] = t_start;
  a->njet += 1;
  return HYDRO_OK;
}

hydro_status hydro_adjoint_set_params(hydro_adjoint* a, double k_rad, double k_coll) {
  if (!a || !std::isfinite(k_rad) || !std::isfinite(k_coll)) return HYDRO_EINVAL;
  a->cfg.k_rad = k_rad;
  a->cfg.k_coll = k_coll;
  a->forward_done = false;
  return HYDRO_OK;
}

hydro_status hydro_adjoint_forward(hydro_adjoint* a, const double* d_prim5, double* J) {
  NvtxRange call("hydro_adjoint_forward");
  if (!a || !d_prim5 || !J) return HYDRO_EINVAL;
  const size_t f5 = 5 * a->n * sizeof(double);
  cudaError_t err = cudaMemcpyAsync(a->prim, d_prim5, f5, cudaMemcpyDeviceToDevice, a->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(a->diag, 0, sizeof(DevDiag), a->stream);
  if (err == cudaSuccess) err = launch_init(HYDRO_FP64, HYDRO_PRIMITIVE, a->prim, a->ckpt[0], a->n, a->diag, a->stream);
  // march segment by segment from each checkpoint, step i of a segment at position
  // i of set 0, the last step of a segment ending in the next checkpoint.  The last
  // segment's states stay in set 0 where the reverse sweep reads them, so that the
  // reverse sweep need not replay it.
  AdjSet& S = a->set[0];
  const double* cur = a->ckpt[0];
  for (int k = 0; k < a->nckpt && err == cudaSuccess; ++k) {
    const int s0 = k * a->every, len = std::min(a->nsteps, s0 + a->every) - s0;
    for (int i = 0; i < len && err == cudaSuccess; ++i) {
      double* out = (i == len - 1 && k + 1 < a->nckpt) ? a->ckpt[k + 1] : S.seg[i + 1];
      err = forward_step(a, s0 + i, S, i, i == 0 ? a->ckpt[k] : S.seg[i], out, a->stream);
      cur = out;
    }
  }
  if (err == cudaSuccess) cone_energy_kernel<<<kConeBlocks, 256, 0, a->stream>>>(cur, a->cone, a->partial);
  std::vector<double> part(kConeBlocks);
  DevDiag d;
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(part.data(), a->partial, kConeBlocks * sizeof(double), cudaMemcpyDeviceToHost, a->stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(&d, a->diag, sizeof(d), cudaMemcpyDeviceToHost, a->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(a->stream);
  if (err != cudaSuccess) return HYDRO_ECUDA;
  if (d.bad_input) return HYDRO_EINVAL;
  if (d.status) return (hydro_status)d.status;
  double sum = 0.0;
  for (double v : part) sum += v;
  a->J = sum;
  *J = sum;
  a->forward_done = true;
  a->last_kept = true;
  return HYDRO_OK;
}

hydro_status hydro_adjoint_backward(hydro_adjoint* a, double dJ, double* grad_k_rad, double* grad_k_coll,
                                    double* d_grad_e) {
  if (!a || !d_grad_e) return HYDRO_EINVAL;
  if (!a->forward_done) return HYDRO_ESTATE;
  NvtxRange call("hydro_adjoint_backward");
  cudaError_t err = cudaMemsetAsync(a->kbar, 0, 2 * kMaxJets * sizeof(double), a->stream);
  // the fields past the combinations' kAdjFields stay zero (the seed zeroes lamA's)
  for (double* l : {a->lamB, a->lam0})
    if (err == cudaSuccess)
      err = cudaMemsetAsync(l + kAdjFields * a->n, 0, (5 - kAdjFields) * a->n * sizeof(double), a->stream);
  if (err == cudaSuccess) {
    cone_seed_kernel<<<grid_1d(a->n), 256, 0, a->stream>>>(a->lamA, a->cone, dJ);
    err = cudaGetLastError();
    if (err == cudaSuccess && a->lamf) {
      scale_to_float_kernel<<<grid_1d(5 * a->n), 256, 0, a->stream>>>(a->lamA, a->lamf, kRK3B[2] * a->cfg.dt, 5 * a->n);
      err = cudaGetLastError();
    }
  }
  // segments in reverse: the step and stage states of a segment are recomputed
  // from its checkpoint into one of two buffer sets on the side stream while the
  // main stream walks the previous segment's steps backwards in the other set
  const bool mixed = a->cfg.precision == HYDRO_MIXED;
  auto set_of = [&](int k) { return (a->nckpt - 1 - k) & 1; };
  auto recompute = [&](int k, cudaStream_t st) {
    const int s0 = k * a->every, len = std::min(a->nsteps, s0 + a->every) - s0;
    AdjSet& S = a->set[set_of(k)];
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < len && e == cudaSuccess; ++i)
      e = forward_step(a, s0 + i, S, i, i == 0 ? a->ckpt[k] : S.seg[i], S.seg[i + 1], st);
    return e;
  };
  const int last = a->nckpt - 1;
  if (err == cudaSuccess && !a->last_kept) err = recompute(last, a->stream);   // set 0
  a->last_kept = false;   // the replays below overwrite the segment buffers
  // the side stream starts after everything issued so far (checkpoints, seeds); set 1 is free
  if (err == cudaSuccess) err = cudaEventRecord(a->ev_start, a->stream);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(a->side, a->ev_start, 0);
  if (err == cudaSuccess) err = cudaEventRecord(a->ev_free[1], a->stream);
  for (int k = last; k >= 0 && err == cudaSuccess; --k) {
    if (k >= 1) {   // refill the other set with segment k - 1 once its previous reader is done
      const int o = set_of(k - 1);
      err = cudaStreamWaitEvent(a->side, a->ev_free[o], 0);
      if (err == cudaSuccess) err = recompute(k - 1, a->side);
      if (err == cudaSuccess) err = cudaEventRecord(a->ev_ready[o], a->side);
    }
    if (err == cudaSuccess && k < last) err = cudaStreamWaitEvent(a->stream, a->ev_ready[set_of(k)], 0);
    const int s0 = k * a->every;
    const int len = std::min(a->nsteps, s0 + a->every) - s0;
    const AdjSet& S = a->set[set_of(k)];
    for (int s = len - 1; s >= 0 && err == cudaSuccess; --s) {
      const int64_t n = s0 + s;
      // the stage states (FP64) or their shadows (mixed) of step n
      auto Uk = [&](int st) -> const double* {
        if (mixed) return nullptr;
        return st == 0 ? (s == 0 ? a->ckpt[k] : S.seg[s]) : S.stages[2 * s + st - 1];
      };
      auto Sk = [&](int st) -> const float* { return mixed ? S.shd[3 * s + st] : nullptr; };
      // stage 3: U = 1/3 U0 + 2/3 (U2 + dt L(U2))
      err = vjp(a, n, 2, Uk(2), Sk(2), a->lamA, kRK3B[2] * a->cfg.dt);
      if (err == cudaSuccess) err = combine(a, 0, 2);
      // stage 2: U2 = 3/4 U0 + 1/4 (U1 + dt L(U1))
      if (err == cudaSuccess) err = vjp(a, n, 1, Uk(1), Sk(1), a->lamB, kRK3B[1] * a->cfg.dt);
      if (err == cudaSuccess) err = combine(a, 1, 1);
      // stage 1: U1 = U0 + dt L(U0)
      if (err == cudaSuccess) err = vjp(a, n, 0, Uk(0), Sk(0), a->lamA, kRK3B[0] * a->cfg.dt);
      if (err == cudaSuccess) err = combine(a, 2, 0);
      std::swap(a->lamA, a->lam0);   // adjoint of the step's input becomes the next output adjoint
    }
    if (err == cudaSuccess) err = cudaEventRecord(a->ev_free[set_of(k)], a->stream);
  }
  if (err == cudaSuccess) {
    grad_e_kernel<<<grid_1d(a->n), 256, 0, a->stream>>>(a->prim, a->lamA, d_grad_e, a->n);
    err = cudaGetLastError();
  }
  double kb[2 * kMaxJets];
  int status = 0;
  if (err == cudaSuccess) err = cudaMemcpyAsync(kb, a->kbar, sizeof(kb), cudaMemcpyDeviceToHost, a->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(&status, &a->diag->status, sizeof(int), cudaMemcpyDeviceToHost, a->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(a->stream);
  if (err != cudaSuccess) return HYDRO_ECUDA;
  if (status) return (hydro_status)status;   // raised by the recomputation or, in the checked build, a check
  double gr = 0.0, gc = 0.0;
  for (int j = 0; j < a->njet; ++j) {
    gr += kb[2 * j];
    gc += kb[2 * j + 1];
  }
  if (grad_k_rad) *grad_k_rad = gr;
  if (grad_k_coll) *grad_k_coll = gc;
  return HYDRO_OK;
}

void hydro_adjoint_destroy(hydro_adjoint* a) {
  if (!a) return;
  if (a->stream || a->ws) cudaStreamSynchronize(a->stream);
  if (a->side) {
    cudaStreamSynchronize(a->side);
    cudaStreamDestroy(a->side);
  }
  for (cudaEvent_t e : {a->ev_start, a->ev_ready[0], a->ev_ready[1], a->ev_free[0], a->ev_free[1]})
    if (e) cudaEventDestroy(e);
  if (a->owns_ws && a->ws) cudaFree(a->ws);
  delete a;
}

}  // extern "C"
