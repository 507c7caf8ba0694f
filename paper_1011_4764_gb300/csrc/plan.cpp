// Host planner: geometry validation, fragment storage table, pair list with
// per-pair overlap geometry, and contraction work items.
//
// Sec. II of the paper keeps the pairs of fragments that are close in space;
// here a pair a <= b is kept exactly when box a meets the dilated box of b,
// the only pairs whose blocks can be non-zero for states confined to their
// boxes.  The overlap region B_a ∩ B_b+ is a product of per-dimension point
// sets; on the periodic grid each is a union of at most a few runs, and each
// product of runs (a "piece") is a box that is contiguous in both fragments'
// storage coordinates.
#include <algorithm>
#include <cstdio>

#include "ofm_internal.h"

namespace ofm {

static inline int pmod(long long a, int n) {
  long long r = a % n;
  return (int)(r < 0 ? r + n : r);
}

std::vector<Run> dim_runs(int n, int offa, int exta, int offb, int extb) {
  std::vector<Run> runs;
  int prev_lb = -2;
  for (int t = 0; t < exta; ++t) {
    int g = pmod((long long)offa + t, n);
    int lb = pmod((long long)g - offb, n);
    if (lb >= extb) {
      prev_lb = -2;
      continue;
    }
    if (!runs.empty() && prev_lb >= 0 && lb == prev_lb + 1 && runs.back().ta + runs.back().len == t) {
      runs.back().len++;
    } else {
      runs.push_back(Run{t, lb, 1});
    }
    prev_lb = lb;
  }
  return runs;
}

static long long dim_count(int n, int offa, int exta, int offb, int extb) {
  long long c = 0;
  for (int t = 0; t < exta; ++t) {
    int lb = pmod((long long)pmod((long long)offa + t, n) - offb, n);
    if (lb < extb) ++c;
  }
  return c;
}

bool validate_geometry(const ofm_grid& g, const ofm_fragment* f, int nf, std::string& err) {
  char buf[256];
  if (!(g.h > 0.0)) { err = "grid spacing h must be > 0"; return false; }
  for (int d = 0; d < 3; ++d)
    if (g.n[d] < 1) { err = "grid dimensions must be >= 1"; return false; }
  if ((long long)g.n[0] * g.n[1] * g.n[2] > (1LL << 31)) { err = "grid has more than 2^31 points"; return false; }
  if (nf < 1 || f == nullptr) { err = "need at least one fragment"; return false; }
  for (int a = 0; a < nf; ++a) {
    long long P = 1;
    for (int d = 0; d < 3; ++d) {
      int e = f[a].ext[d];
      if (e < 1 || e > g.n[d]) {
        snprintf(buf, sizeof buf, "fragment %d: ext[%d]=%d outside [1, %d]", a, d, e, g.n[d]);
        err = buf; return false;
      }
      if (e == g.n[d] - 1) {
        snprintf(buf, sizeof buf, "fragment %d: ext[%d]=%d equals n-1; its dilated box would wrap onto itself", a, d, e);
        err = buf; return false;
      }
      P *= e;
    }
    long long Pd = 1;
    for (int d = 0; d < 3; ++d) Pd *= (f[a].ext[d] < g.n[d]) ? f[a].ext[d] + 2 : f[a].ext[d];
    if (Pd * 1024 >= (1LL << 31)) {
      snprintf(buf, sizeof buf, "fragment %d: box of %lld points is too large (limit 2^21)", a, Pd);
      err = buf; return false;
    }
    if (f[a].n_states < 1 || f[a].n_states > P - 1 || f[a].n_states > 1024) {
      snprintf(buf, sizeof buf, "fragment %d: n_states=%d outside [1, min(P-1, 1024)] (P=%lld)", a,
               f[a].n_states, P);
      err = buf; return false;
    }
  }
  return true;
}

void make_frag_table(const ofm_grid& g, const ofm_fragment* f, int nf, std::vector<DevFrag>& out,
                     long long& total_elems) {
  out.assign(nf, DevFrag{});
  long long off = 0;
  int basis = 0;
  for (int a = 0; a < nf; ++a) {
    DevFrag& r = out[a];
    r.Pd = 1;
    for (int d = 0; d < 3; ++d) {
      r.ext[d] = f[a].ext[d];
      r.full[d] = (f[a].ext[d] == g.n[d]) ? 1 : 0;
      if (r.full[d]) {
        r.doff[d] = pmod(f[a].off[d], g.n[d]);
        r.dext[d] = g.n[d];
        r.lo[d] = 0;
      } else {
        r.doff[d] = pmod((long long)f[a].off[d] - 1, g.n[d]);
        r.dext[d] = f[a].ext[d] + 2;
        r.lo[d] = 1;
      }
      r.Pd *= r.dext[d];
    }
    r.n = f[a].n_states;
    r.ld = (r.n + 3) / 4 * 4;
    r.basis0 = basis;
    basis += r.n;
    r.off = off;
    off += (r.Pd * r.ld + 63) / 64 * 64;
  }
  total_elems = off;
}

void make_pairs(const ofm_grid& g, const std::vector<DevFrag>& fr, std::vector<HostPair>& pairs) {
  pairs.clear();
  const int nf = (int)fr.size();
  for (int a = 0; a < nf; ++a) {
    const DevFrag& A = fr[a];
    int offa[3];
    for (int d = 0; d < 3; ++d) offa[d] = pmod((long long)A.doff[d] + A.lo[d], g.n[d]);
    for (int b = a; b < nf; ++b) {
      const DevFrag& B = fr[b];
      std::vector<Run> runs[3];
      bool meet = true;
      for (int d = 0; d < 3 && meet; ++d) {
        runs[d] = dim_runs(g.n[d], offa[d], A.ext[d], B.doff[d], B.dext[d]);
        meet = !runs[d].empty();
      }
      if (!meet) continue;
      HostPair hp;
      hp.a = a;
      hp.b = b;
      hp.kh = 1;
      hp.ks = 1;
      for (int d = 0; d < 3; ++d) {
        long long s = 0;
        for (auto& r : runs[d]) s += r.len;
        hp.kh *= s;
        int offb = pmod((long long)B.doff[d] + B.lo[d], g.n[d]);
        hp.ks *= dim_count(g.n[d], offa[d], A.ext[d], offb, B.ext[d]);
      }
      for (auto& rz : runs[2])
        for (auto& ry : runs[1])
          for (auto& rx : runs[0]) {
            Piece p;
            p.la[0] = A.lo[0] + rx.ta; p.la[1] = A.lo[1] + ry.ta; p.la[2] = A.lo[2] + rz.ta;
            p.lb[0] = rx.lb; p.lb[1] = ry.lb; p.lb[2] = rz.lb;
            p.len[0] = rx.len; p.len[1] = ry.len; p.len[2] = rz.len;
            hp.pieces.push_back(p);
          }
      pairs.push_back(std::move(hp));
    }
  }
}

void make_items_simt(const std::vector<DevFrag>& fr, const std::vector<HostPair>& pairs, int tile,
                     long long chunk, std::vector<DevPair>& dpairs, std::vector<Piece>& pieces,
                     std::vector<WorkItem>& items, long long& partial_elems) {
  dpairs.clear();
  pieces.clear();
  items.clear();
  partial_elems = 0;
  long long blk = 0;
  for (int p = 0; p < (int)pairs.size(); ++p) {
    const HostPair& hp = pairs[p];
    const DevFrag& A = fr[hp.a];
    const DevFrag& B = fr[hp.b];
    DevPair dp;
    dp.a = hp.a;
    dp.b = hp.b;
    dp.mtiles = (A.n + tile - 1) / tile;
    dp.ntiles = (2 * B.n + tile - 1) / tile;
    dp.blk_off = blk;
    blk += 2LL * A.n * B.n;
    // K chunks: whole rows of each piece
    struct Chunk { int piece, r0, r1; };
    std::vector<Chunk> chunks;
    for (const Piece& pc : hp.pieces) {
      int pid = (int)pieces.size();
      pieces.push_back(pc);
      int rows = pc.len[1] * pc.len[2];
      int per = (int)std::max<long long>(1, chunk / pc.len[0]);
      for (int r0 = 0; r0 < rows; r0 += per) chunks.push_back({pid, r0, std::min(rows, r0 + per)});
    }
    dp.nchunk = (int)chunks.size();
    dp.item0 = (int)items.size();
    for (int mt = 0; mt < dp.mtiles; ++mt)
      for (int nt = 0; nt < dp.ntiles; ++nt)
        for (const Chunk& c : chunks) {
          WorkItem w;
          w.pair = p;
          w.piece = c.piece;
          w.r0 = c.r0;
          w.r1 = c.r1;
          w.mt = mt;
          w.nt = nt;
          w.part_off = partial_elems;
          partial_elems += (long long)tile * tile;
          items.push_back(w);
        }
    dp.nitem = (int)items.size() - dp.item0;
    dpairs.push_back(dp);
  }
}

}  // namespace ofm

extern "C" ofm_status ofm_plan_pairs(const ofm_grid* grid, const ofm_fragment* frags, int n_frag,
                                     int* n_pairs, int* pair_ab, long long* counts, int max_pairs,
                                     long long* pair_flops) {
  if (!grid || !frags || !n_pairs) return OFM_ERR_INVALID;
  std::string err;
  if (!ofm::validate_geometry(*grid, frags, n_frag, err)) return OFM_ERR_INVALID;
  std::vector<ofm::DevFrag> fr;
  long long tot = 0;
  ofm::make_frag_table(*grid, frags, n_frag, fr, tot);
  std::vector<ofm::HostPair> pairs;
  ofm::make_pairs(*grid, fr, pairs);
  *n_pairs = (int)pairs.size();
  long long F = 0;
  for (size_t i = 0; i < pairs.size(); ++i) {
    const auto& p = pairs[i];
    F += 2LL * fr[p.a].n * fr[p.b].n * (p.ks + p.kh);
    if ((int)i < max_pairs) {
      if (pair_ab) {
        pair_ab[2 * i] = p.a;
        pair_ab[2 * i + 1] = p.b;
      }
      if (counts) {
        counts[2 * i] = p.ks;
        counts[2 * i + 1] = p.kh;
      }
    }
  }
  if (pair_flops) *pair_flops = F;
  return OFM_OK;
}
