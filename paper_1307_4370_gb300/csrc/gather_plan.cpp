// Host-side plan of G and G^T (see gather_plan.h).
#include "gather_plan.h"

#include <algorithm>
#include <utility>

namespace purify {

int build_gather_plan(const int* k0, const GatherPlanParams& prm, GatherPlan& out) {
  const int64_t M = prm.M;
  const int T = prm.T, J = prm.J, L = prm.L, NT = kGridThreads;
  if (M < 0 || T < 2 || (T & (T - 1)) != 0 || T > 64 || L % T != 0 || J < 2 || J > 8 || J > L ||
      prm.entry_bytes == 0 || prm.tab_stride < (T / 2) * (T / 2) + 1 || prm.max_partials < 2)
    return -1;
  const int TD = L / T, ntiles = TD * TD;
  out = GatherPlan{};
  out.ntiles = ntiles;
  out.tiles_1d = TD;
  auto kr_of = [&](int64_t i) { return k0[2 * i]; };
  auto kc_of = [&](int64_t i) { return k0[2 * i + 1]; };
  for (int64_t i = 0; i < M; ++i)
    if (kr_of(i) < 0 || kr_of(i) >= L || kc_of(i) < 0 || kc_of(i) >= L) return -1;

  // counting sort by home tile (stable: keeps the caller's order inside a tile)
  std::vector<int>& cnt = out.home;
  cnt.assign(ntiles + 1, 0);
  out.perm.resize(M);
  for (int64_t i = 0; i < M; ++i) cnt[(kr_of(i) / T) * TD + kc_of(i) / T + 1]++;
  for (int t = 0; t < ntiles; ++t) cnt[t + 1] += cnt[t];
  {
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < M; ++i) out.perm[pos[(kr_of(i) / T) * TD + kc_of(i) / T]++] = (int)i;
  }

  // per-tile lists of sorted indices whose footprint meets the tile
  auto tiles_of = [&](int64_t si, int* tl) {
    const int64_t i = out.perm[si];
    const int r0 = kr_of(i) / T, r1 = ((kr_of(i) + J - 1) % L) / T;
    const int c0 = kc_of(i) / T, c1 = ((kc_of(i) + J - 1) % L) / T;
    int nt = 0;
    const int rs[2] = {r0, r1}, cs[2] = {c0, c1};
    for (int a = 0; a < (r1 != r0 ? 2 : 1); ++a)
      for (int b = 0; b < (c1 != c0 ? 2 : 1); ++b) tl[nt++] = rs[a] * TD + cs[b];
    return nt;
  };
  // (list positions are 32-bit on the device: at most 2^31 - 1 entries)
  std::vector<int64_t> lcnt64(ntiles + 1, 0);
  int tl[4];
  for (int64_t si = 0; si < M; ++si) {
    const int nt = tiles_of(si, tl);
    for (int k = 0; k < nt; ++k) lcnt64[tl[k] + 1]++;
  }
  for (int t = 0; t < ntiles; ++t) lcnt64[t + 1] += lcnt64[t];
  const int64_t nlist = lcnt64[ntiles];
  if (nlist > 0x7fffffff) return -2;
  std::vector<int>& lcnt = out.list_off;
  lcnt.assign(lcnt64.begin(), lcnt64.end());
  out.list.resize(nlist);
  out.lkey.resize(nlist);
  {
    std::vector<int> pos(lcnt.begin(), lcnt.end() - 1);
    for (int64_t si = 0; si < M; ++si) {
      const int nt = tiles_of(si, tl);
      for (int k = 0; k < nt; ++k) out.list[pos[tl[k]]++] = (int)si;
    }
  }
  // order each tile's list by the footprint start cell relative to the tile:
  // the visibilities starting at a given cell form one run
  const int W = T + J - 1;
  auto rel = [&](int k, int origin) {  // start offset in [-(J-1), L - J + 1)
    int t = (k - origin) % L;
    if (t < 0) t += L;
    return t >= L - (J - 1) ? t - L : t;
  };
  {
    std::vector<std::pair<int, int>> seg;
    for (int t = 0; t < ntiles; ++t) {
      const int R0 = (t / TD) * T, C0 = (t % TD) * T;
      seg.clear();
      for (int e = lcnt[t]; e < lcnt[t + 1]; ++e) {
        const int64_t i = out.perm[out.list[e]];
        const int key = (rel(kr_of(i), R0) + J - 1) * W + (rel(kc_of(i), C0) + J - 1);
        seg.emplace_back(key, out.list[e]);
      }
      std::stable_sort(seg.begin(), seg.end(),
                       [](const std::pair<int, int>& x, const std::pair<int, int>& y) { return x.first < y.first; });
      for (size_t k = 0; k < seg.size(); ++k) {
        out.list[lcnt[t] + k] = seg[k].second;
        out.lkey[lcnt[t] + k] = seg[k].first;
      }
    }
  }

  // gridding work units: each tile's list in chunks whose entries, with the
  // kernel's fixed tables, fit the shared-memory budget (large tiles: room
  // for at least 256 entries beyond the fixed part)
  const int64_t mean = (nlist + ntiles - 1) / ntiles;
  const int64_t fixed = (int64_t)prm.fixed_bytes, per = (int64_t)prm.entry_bytes;
  const int64_t budget = std::max<int64_t>((int64_t)prm.smem_budget, fixed + 256 * per);
  const int cap = (int)std::max<int64_t>(128, (budget - fixed) / per / 32 * 32);
  out.chunk_max = (int)std::min<int64_t>(cap, std::max<int64_t>(256, ((3 * mean / 2 + 127) / 128) * 128));
  out.slot0.assign(ntiles, -1);
  out.nchunk.assign(ntiles, 0);
  for (int t = 0; t < ntiles; ++t) {
    const int b = lcnt[t], e = lcnt[t + 1];
    const int nc = std::max(1, (e - b + out.chunk_max - 1) / out.chunk_max);
    out.nchunk[t] = nc;
    if (nc > 1) out.slot0[t] = out.nslots;
    for (int k = 0; k < nc; ++k) {
      const int cb = b + (int)((int64_t)(e - b) * k / nc), ce = b + (int)((int64_t)(e - b) * (k + 1) / nc);
      out.chunks.push_back(PlanI4{t, cb, ce, nc > 1 ? out.nslots + k : -1});
    }
    if (nc > 1) out.nslots += nc;
  }
  // heavy chunks first
  std::stable_sort(out.chunks.begin(), out.chunks.end(),
                   [](const PlanI4& a, const PlanI4& b) { return a.z - a.y > b.z - b.y; });
  const int nchunks = (int)out.chunks.size();

  // per chunk, the gather's walk (it depends on the frequencies only): the
  // prefix P[o] of the owners' work (2 x 2 cell blocks, o = 0..NO) as 16-bit
  // values, and the items of the steps of each thread's slice, step-major
  const int NK = W * W, HB = T / 2, NO = HB * HB;
  if (out.chunk_max > (1 << kItemEntryBits) || NO > 1024) return -2;
  out.tab.assign((size_t)nchunks * prm.tab_stride, 0);
  out.item_row.assign(nchunks, 0);
  std::vector<int> off(NK + 1);
  int64_t rows = 0;
  for (int q = 0; q < nchunks; ++q) {
    const PlanI4 ch = out.chunks[q];
    const int* kb = out.lkey.data() + ch.y;
    const int ne = ch.z - ch.y;
    // off[k] = first entry with start-cell key >= k (k = 0..NK)
    for (int k = 0, e = 0; k <= NK; ++k) {
      while (e < ne && kb[e] < k) ++e;
      off[k] = e;
    }
    uint16_t* t = out.tab.data() + (size_t)q * prm.tab_stride;
    int acc = 0;
    for (int o = 0; o < NO; ++o) {
      t[o] = (uint16_t)acc;
      const int R = 2 * (o / HB), C = 2 * (o % HB);
      for (int kr = R; kr <= R + J; ++kr) acc += off[kr * W + C + J + 1] - off[kr * W + C];
    }
    t[NO] = (uint16_t)acc;
    if (acc > 65535) return -2;  // not reachable with chunk_max <= 864 (<= 25 owners per entry)
    // thread j walks steps [t0(j), t0(j + 1)) of the owners' concatenated runs
    const int Wt = acc;
    const int64_t nrow = (Wt + NT - 1) / NT;
    out.item_row[q] = (int)rows;
    out.items.resize((size_t)(rows + nrow) * NT, 0u);
    uint32_t* dst = out.items.data() + (size_t)rows * NT;
    rows += nrow;
    auto t0_of = [&](int jj) { return (int)(((int64_t)jj * Wt + NT - 1) / NT); };
    int jj = 0, tj0 = 0, tj1 = t0_of(1), tt = 0;
    for (int o = 0; o < NO; ++o) {
      const int R = 2 * (o / HB), C = 2 * (o % HB);
      for (int kr = R; kr <= R + J; ++kr) {
        for (int e = off[kr * W + C]; e < off[kr * W + C + J + 1]; ++e, ++tt) {
          while (tt >= tj1) {
            ++jj;
            tj0 = tj1;
            tj1 = t0_of(jj + 1);
          }
          const int kc = kb[e] - kr * W;  // start column, in [C, C + J]
          dst[(size_t)(tt - tj0) * NT + jj] = grid_item(e, R + J - kr, C + J - kc, o);
        }
      }
    }
  }
  out.nitem_rows = rows;
  if (rows > 0x7fffffff) return -2;

  // degridding work units: each tile's home visibilities (a run of the sorted
  // order) in chunks of at most dch; dch keeps the number of chunks (one FP64
  // partial-sum slot each) within max_partials: at most ntiles + M / dch
  const int64_t dch = std::max<int64_t>(1024, (2 * M + prm.max_partials - 1) / prm.max_partials);
  for (int t = 0; t < ntiles; ++t) {
    const int b = cnt[t], e = cnt[t + 1];
    const int nc = (int)((e - b + dch - 1) / dch);
    for (int k = 0; k < nc; ++k) {
      const int cb = b + (int)((int64_t)(e - b) * k / nc), ce = b + (int)((int64_t)(e - b) * (k + 1) / nc);
      out.dchunks.push_back(PlanI4{t, cb, ce, 0});
    }
  }
  std::stable_sort(out.dchunks.begin(), out.dchunks.end(),
                   [](const PlanI4& a, const PlanI4& b) { return a.z - a.y > b.z - b.y; });
  return 0;
}

}  // namespace purify
