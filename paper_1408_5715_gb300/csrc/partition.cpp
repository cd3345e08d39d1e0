// partition.cpp -- splitting a mesh into parts for several processes.
//
// Part p of P owns the contiguous range [p*n/P, (p+1)*n/P) of the current
// cell numbering (after RCM or Hilbert renumbering these ranges are compact
// regions, so halos are small).  Its local numbering lists the owned cells
// first, in global order, then the halo: every cell outside the part that an
// owned cell has as a neighbour, in ascending global id.  The local neighbour
// table indexes that local numbering (ghost-face codes stay negative), so a
// part can be stepped like a mesh whose halo states are refreshed from their
// owners after every stage, with the CFL minimum reduced over all parts.
#include <algorithm>

#include "fv_internal.h"

namespace fv {

PartRange part_range(int64_t n, int32_t nparts, int32_t part) {
  if (nparts < 1 || part < 0 || part >= nparts) throw Error{FV_EINVAL, "bad part index"};
  PartRange r;
  r.begin = n * part / nparts;
  r.end = n * (part + 1) / nparts;
  return r;
}

LocalPart build_local_part(const HostMesh& m, int32_t nparts, int32_t part) {
  const PartRange r = part_range(m.n, nparts, part);
  LocalPart lp;
  lp.n_owned = r.end - r.begin;
  std::vector<int64_t> halo;
  for (int64_t c = r.begin; c < r.end; ++c)
    for (int k = 0; k < 3; ++k) {
      const int32_t x = m.nbr[3 * c + k];
      if (x >= 0 && (x < r.begin || x >= r.end)) halo.push_back(x);
    }
  std::sort(halo.begin(), halo.end());
  halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
  lp.global.resize(lp.n_owned + halo.size());
  for (int64_t c = 0; c < lp.n_owned; ++c) lp.global[c] = r.begin + c;
  for (size_t j = 0; j < halo.size(); ++j) lp.global[lp.n_owned + j] = halo[j];
  lp.halo_owner.resize(halo.size());
  for (size_t j = 0; j < halo.size(); ++j) {
    // owner of a global id: the part whose range contains it
    int32_t p = (int32_t)((halo[j] * nparts) / std::max<int64_t>(m.n, 1));
    while (p > 0 && halo[j] < part_range(m.n, nparts, p).begin) --p;
    while (p + 1 < nparts && halo[j] >= part_range(m.n, nparts, p).end) ++p;
    lp.halo_owner[j] = p;
  }
  lp.nbr.resize(3 * lp.n_owned);
  lp.nrm.resize(6 * lp.n_owned);
  lp.vol.resize(lp.n_owned);
  for (int64_t c = 0; c < lp.n_owned; ++c) {
    const int64_t g = r.begin + c;
    for (int k = 0; k < 3; ++k) {
      const int32_t x = m.nbr[3 * g + k];
      int32_t loc = x;
      if (x >= r.begin && x < r.end) {
        loc = (int32_t)(x - r.begin);
      } else if (x >= 0) {
        loc = (int32_t)(lp.n_owned +
                        (std::lower_bound(halo.begin(), halo.end(), (int64_t)x) - halo.begin()));
      }
      lp.nbr[3 * c + k] = loc;
    }
    for (int k = 0; k < 6; ++k) lp.nrm[6 * c + k] = m.nrm[6 * g + k];
    lp.vol[c] = m.vol[g];
  }
  return lp;
}

}  // namespace fv
