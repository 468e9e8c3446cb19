// Host-only entry points of the C ABI: error reporting and planner
// introspection (no CUDA calls; usable on a machine without a GPU).
#include <cstring>
#include <string>
#include <utility>

#include "../../include/dmrg_gb300.h"
#include "plan.hpp"

namespace dmrg {
thread_local std::string g_last_error;
void set_error(const std::string &s) { g_last_error = s; }
}  // namespace dmrg

extern "C" const char *dmrg_last_error(void) { return dmrg::g_last_error.c_str(); }

static dmrg::Integrals make_integrals(int L, const double *h, const double *v) {
  dmrg::Integrals I;
  I.L = L;
  I.h.assign(h, h + (size_t)L * L);
  I.v.assign(v, v + (size_t)L * L * L * L);
  return I;
}

static int copy_out(const std::string &s, char *buf, long long buflen, long long *needed) {
  if (needed) *needed = (long long)s.size() + 1;
  if (!buf || buflen < (long long)s.size() + 1) {
    dmrg::set_error("dump buffer too small");
    return buf ? DMRG_EINVAL : DMRG_OK;
  }
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return DMRG_OK;
}

extern "C" int dmrg_debug_pieces(int L, const double *h, const double *v, int k, int l_empty,
                                 int r_empty, int compress, char *buf, long long buflen,
                                 long long *needed) {
  try {
    if (L < 2 || k < 0 || k > L - 2 || !h || !v) {
      dmrg::set_error("dmrg_debug_pieces: bad arguments");
      return DMRG_EINVAL;
    }
    auto I = make_integrals(L, h, v);
    auto ps = dmrg::hamiltonian_pieces(I, k, l_empty != 0, r_empty != 0);
    if (compress) ps = dmrg::compress_pieces(std::move(ps));
    return copy_out(dmrg::dump_pieces(ps), buf, buflen, needed);
  } catch (const std::exception &e) {
    dmrg::set_error(e.what());
    return DMRG_EINVAL;
  }
}

extern "C" int dmrg_debug_newops(int L, const double *h, const double *v, int k, int side,
                                 int old_empty, char *buf, long long buflen, long long *needed) {
  try {
    if (L < 2 || k < 0 || k > L - 2 || (side != 0 && side != 1) || !h || !v) {
      dmrg::set_error("dmrg_debug_newops: bad arguments");
      return DMRG_EINVAL;
    }
    auto I = make_integrals(L, h, v);
    dmrg::BlockLayout nb;
    std::vector<int> sites;
    if (side == 0) for (int s = 0; s <= k; ++s) sites.push_back(s);
    else for (int s = k + 1; s < L; ++s) sites.push_back(s);
    dmrg::build_layout(nb, side, L, sites, {{0, 0, 1}});
    auto ops = dmrg::new_block_ops(I, k, side, nb, old_empty != 0);
    std::string out;
    for (auto &o : ops) {
      const auto &F = nb.fam[o.fam];
      out += "OP " + std::to_string(F.kind) + " " + std::to_string(F.idx[o.k][0]) + " " +
             std::to_string(F.idx[o.k][1]) + "\n";
      out += dmrg::dump_halfop(o.def);
    }
    return copy_out(out, buf, buflen, needed);
  } catch (const std::exception &e) {
    dmrg::set_error(e.what());
    return DMRG_EINVAL;
  }
}

extern "C" int dmrg_debug_truncation(int nsectors, const int *dims, const double *ev_ascending, int mkeep,
                                     int *kept, int *cols, double *out3) {
  try {
    if (nsectors < 0 || mkeep < 0 || (nsectors > 0 && (!dims || !kept)) || !out3) {
      dmrg::set_error("dmrg_debug_truncation: bad arguments");
      return DMRG_EINVAL;
    }
    std::vector<std::vector<double>> ev(nsectors);
    long long pos = 0;
    for (int e = 0; e < nsectors; ++e) {
      if (dims[e] < 0) {
        dmrg::set_error("dmrg_debug_truncation: negative sector dimension");
        return DMRG_EINVAL;
      }
      if (dims[e] > 0 && !ev_ascending) {
        dmrg::set_error("dmrg_debug_truncation: NULL eigenvalues");
        return DMRG_EINVAL;
      }
      ev[e].assign(ev_ascending + pos, ev_ascending + pos + dims[e]);
      pos += dims[e];
    }
    const dmrg::KeptSet ks = dmrg::choose_kept(ev, mkeep, 1e-13);
    long long c = 0;
    for (int e = 0; e < nsectors; ++e) {
      kept[e] = ks.kept[e];
      for (int j : ks.cols[e]) {
        if (cols) cols[c] = j;
        ++c;
      }
    }
    out3[0] = ks.trace;
    out3[1] = ks.kept_weight;
    out3[2] = ks.cut_gap;
    return DMRG_OK;
  } catch (const std::exception &e) {
    dmrg::set_error(e.what());
    return DMRG_EINVAL;
  }
}

extern "C" int dmrg_debug_pair_rdm(int nblocks, const int *abcd, const long long *off_size, const double *psi,
                                   double *rho2, double *s3) {
  try {
    if (nblocks < 1 || !abcd || !off_size || !psi) {
      dmrg::set_error("dmrg_debug_pair_rdm: bad arguments");
      return DMRG_EINVAL;
    }
    std::vector<dmrg::PsiBlockRef> blocks((size_t)nblocks);
    for (int i = 0; i < nblocks; ++i) {
      const int *q = abcd + 4 * i;
      if (q[1] < 0 || q[1] > 3 || q[2] < 0 || q[2] > 3 || off_size[2 * i] < 0 || off_size[2 * i + 1] < 0) {
        dmrg::set_error("dmrg_debug_pair_rdm: site state outside 0..3 or negative offset/size");
        return DMRG_EINVAL;
      }
      blocks[(size_t)i] = {q[0], q[1], q[2], q[3], (int64_t)off_size[2 * i], (int64_t)off_size[2 * i + 1]};
    }
    double rho[256];
    dmrg::pair_rdm(blocks, psi, rho);
    if (rho2)
      for (int i = 0; i < 256; ++i) rho2[i] = rho[i];
    if (s3) dmrg::orbital_entropies(rho, s3);
    return DMRG_OK;
  } catch (const std::exception &e) {
    dmrg::set_error(e.what());
    return DMRG_EINVAL;
  }
}
