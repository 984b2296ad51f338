// Bounds checks of the sweep tiles and of the adjoint's reverse sweeps, compiled
// in with -DHYDRO_CHECK (the library libhydro_check.so that build.build_checked()
// makes) as a stand-in for a memory checker.  Every global-memory access of a
// tile is q N + o for a field q below the buffer's field count (5, or 6 for the
// mixed shadow) and a cell offset o, so checking o < N at the places a tile forms
// it bounds every access; TMA copies are checked against the copy rules
// (innermost coordinate a multiple of 16 bytes; stores from non-negative
// coordinates).  A failed check records its site and the offending value in the
// diagnostics block, sets HYDRO_ECHECK, and keeps the access inside its buffer
// (the offset is redirected to the last allowed cell) or skips the copy (its
// bounded wait then runs out).  Shared-memory indices are not checked here: they
// follow from the compile-time tile layout.  In the regular build the checks
// compile to nothing.
#pragma once

#include "hydro_internal.h"

namespace hydro {

// hydro_diag.check_site values.
enum CheckSite : int {
  kSiteOperands = 1,   // phase 0: cell offset of the per-thread copies of the accumulator and U0
  kSiteStaging = 2,    // phase 1: cell offset of a staged cell (state, shadow, primitive cache)
  kSiteUpdate = 3,     // phase 3: cell offset of an updated cell (accumulator, result, shadow, jet)
  kSiteTmaLoad = 4,    // a TMA load whose innermost coordinate is not at a 16-byte offset
  kSiteTmaStore = 5,   // a TMA store from such a coordinate or from a negative one
  kSiteAdjWindow = 6,  // adjoint reverse sweep: cell offset of a window position (adjoint, state, r)
  kSiteAdjResult = 7,  // adjoint reverse sweep: cell offset of an updated cell's result
  kSiteAdjJet = 8,     // adjoint reverse sweep: the jet cell's offset
};

#ifdef HYDRO_CHECK
__device__ __forceinline__ void check_failed(DevDiag* d, int site, unsigned value) {
  if (atomicCAS(&d->check_site, 0, site) == 0) d->check_index = value;
  atomicCAS(&d->status, 0, (int)HYDRO_ECHECK);
}

// Cell offset o of a grid of n cells (half of them under the test hook): o, or
// after recording the failure the last allowed offset.
__device__ __forceinline__ unsigned checked_cell(unsigned o, unsigned n, int tighten, int site, DevDiag* d) {
  const unsigned lim = tighten ? (n + 1) / 2 : n;
  if (o < lim) return o;
  check_failed(d, site, o);
  return lim - 1;
}

// Whether a TMA copy with innermost coordinate x (elements of esize bytes) and
// outer coordinates c1, c2 may be issued.
__device__ __forceinline__ bool checked_tma(int x, int esize, int c1, int c2, bool store, DevDiag* d) {
  const bool ok = ((long long)x * esize) % 16 == 0 && (!store || (x >= 0 && c1 >= 0 && c2 >= 0));
  if (!ok) check_failed(d, store ? kSiteTmaStore : kSiteTmaLoad, (unsigned)x);
  return ok;
}

#define HYDRO_CELL_AT(o, n, site, tighten, diag) ::hydro::checked_cell((o), (n), (tighten), (site), (diag))
#define HYDRO_TMA_OK(x, esize, c1, c2, store) ::hydro::checked_tma((x), (esize), (c1), (c2), (store), a.diag)
#else
#define HYDRO_CELL_AT(o, n, site, tighten, diag) (o)
#define HYDRO_TMA_OK(x, esize, c1, c2, store) true
#endif
// the sweep tiles' form: the grid arguments `a` carry the diagnostics block and the test hook
#define HYDRO_CELL(o, n, site) HYDRO_CELL_AT((o), (n), (site), a.check_tighten, a.diag)

}  // namespace hydro
