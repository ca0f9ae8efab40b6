// Host check of the gridding plan (csrc/gather_plan.cpp), no GPU needed.
//
// For seeded footprint start cells it checks the sort, the tile lists, the
// work units and the stored gather walk against brute force, and checks the
// walk's meaning: summing, per chunk, each item's 2 x 2 contribution (the
// kernel's arithmetic, in double) must give the adjoint of interpolation
// G^T y computed by scattering each visibility's J x J footprint (§5).
//
// usage: gather_plan_check L J T M layout seed   (prints "ok" or the failure)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "gather_plan.h"

using namespace purify;

#define CHECK(cond, ...)                    \
  do {                                      \
    if (!(cond)) {                          \
      std::printf("FAIL %s: ", #cond);      \
      std::printf(__VA_ARGS__);             \
      std::printf("\n");                    \
      return 1;                             \
    }                                       \
  } while (0)

int main(int argc, char** argv) {
  if (argc != 7) return 2;
  const int L = std::atoi(argv[1]), J = std::atoi(argv[2]), T = std::atoi(argv[3]);
  const int64_t M = std::atoll(argv[4]);
  const int layout = std::atoi(argv[5]);
  std::mt19937_64 rng(std::strtoull(argv[6], nullptr, 10));
  std::uniform_int_distribution<int> cell(0, L - 1);
  std::uniform_real_distribution<double> unif(-1.0, 1.0);

  // footprint start cells: 0 uniform; 1 half of them on three cells (dense
  // tracks) and the rest uniform; 2 next to the grid's wrap-around edges
  std::vector<int> k0(2 * M);
  const int hot[3][2] = {{cell(rng), cell(rng)}, {cell(rng), cell(rng)}, {L - 1, L - J / 2}};
  for (int64_t i = 0; i < M; ++i) {
    int r = cell(rng), c = cell(rng);
    if (layout == 1 && (i & 1)) {
      r = hot[i % 3][0];
      c = hot[i % 3][1];
    } else if (layout == 2) {
      r = (L - J + (r % (2 * J))) % L;
      c = (L - J + (c % (2 * J))) % L;
    }
    k0[2 * i] = r;
    k0[2 * i + 1] = c;
  }

  GatherPlanParams prm{};
  prm.M = M;
  prm.L = L;
  prm.J = J;
  prm.T = T;
  const int NO = (T / 2) * (T / 2), W = T + J - 1, NT = kGridThreads;
  prm.entry_bytes = 8 + 4 * (2 * (J + 2) + 1);
  prm.fixed_bytes = 16384 + (NO + 1) * 4;
  prm.smem_budget = 72 * 1024;
  prm.tab_stride = (NO + 1 + 7) / 8 * 8;
  prm.max_partials = 32768;
  GatherPlan p;
  const int rc = build_gather_plan(k0.data(), prm, p);
  CHECK(rc == 0, "build_gather_plan returned %d", rc);
  const int TD = L / T, ntiles = TD * TD;
  CHECK(p.ntiles == ntiles && p.tiles_1d == TD, "tiles");
  auto home_tile = [&](int64_t i) { return (k0[2 * i] / T) * TD + k0[2 * i + 1] / T; };

  // sort by home tile, stable
  std::vector<char> seen(M, 0);
  CHECK((int64_t)p.perm.size() == M, "perm size");
  for (int64_t si = 0; si < M; ++si) {
    const int i = p.perm[si];
    CHECK(i >= 0 && i < M && !seen[i], "perm entry %lld", (long long)si);
    seen[i] = 1;
    if (si > 0) {
      const int a = home_tile(p.perm[si - 1]), b = home_tile(i);
      CHECK(a < b || (a == b && p.perm[si - 1] < i), "sorted order at %lld", (long long)si);
    }
  }
  CHECK((int)p.home.size() == ntiles + 1 && p.home[0] == 0 && p.home[ntiles] == M, "home offsets");
  for (int t = 0; t < ntiles; ++t)
    for (int si = p.home[t]; si < p.home[t + 1]; ++si) CHECK(home_tile(p.perm[si]) == t, "home run of tile %d", t);

  // tile lists: exactly the visibilities whose footprint meets the tile, by key
  auto rel = [&](int k, int origin) {
    int d = ((k - origin) % L + L) % L;
    return d >= L - (J - 1) ? d - L : d;
  };
  CHECK((int)p.list_off.size() == ntiles + 1, "list offsets");
  for (int t = 0; t < ntiles; ++t) {
    const int R0 = (t / TD) * T, C0 = (t % TD) * T;
    std::vector<int> want;
    for (int64_t si = 0; si < M; ++si) {
      const int i = p.perm[si];
      bool meets = false;
      for (int a = 0; a < J && !meets; ++a)
        for (int b = 0; b < J && !meets; ++b) {
          const int r = (k0[2 * i] + a) % L, c = (k0[2 * i + 1] + b) % L;
          meets = r >= R0 && r < R0 + T && c >= C0 && c < C0 + T;
        }
      if (meets) want.push_back((int)si);
    }
    const int b = p.list_off[t], e = p.list_off[t + 1];
    CHECK(e - b == (int)want.size(), "tile %d lists %d entries, want %zu", t, e - b, want.size());
    std::vector<int> got(p.list.begin() + b, p.list.begin() + e);
    std::vector<int> gs = got;
    std::sort(gs.begin(), gs.end());
    CHECK(gs == want, "tile %d list members", t);
    for (int k = b; k < e; ++k) {
      const int i = p.perm[p.list[k]];
      const int dr = rel(k0[2 * i], R0), dc = rel(k0[2 * i + 1], C0);
      CHECK(dr >= -(J - 1) && dr < T && dc >= -(J - 1) && dc < T, "start offset in tile %d", t);
      CHECK(p.lkey[k] == (dr + J - 1) * W + (dc + J - 1), "key of entry %d", k);
      if (k > b) CHECK(p.lkey[k - 1] < p.lkey[k] || (p.lkey[k - 1] == p.lkey[k] && p.list[k - 1] < p.list[k]),
                       "list order at %d", k);
    }
  }

  // gridding work units: each tile's list cut into contiguous chunks
  const int nchunks = (int)p.chunks.size();
  CHECK(p.chunk_max >= 1 && p.chunk_max <= (1 << kItemEntryBits), "chunk_max %d", p.chunk_max);
  std::vector<std::vector<PlanI4>> of_tile(ntiles);
  for (int q = 0; q < nchunks; ++q) {
    const PlanI4 ch = p.chunks[q];
    CHECK(ch.x >= 0 && ch.x < ntiles && ch.z - ch.y <= p.chunk_max, "chunk %d", q);
    if (q > 0) CHECK(p.chunks[q - 1].z - p.chunks[q - 1].y >= ch.z - ch.y, "heavy chunks first at %d", q);
    of_tile[ch.x].push_back(ch);
  }
  int slots = 0;
  for (int t = 0; t < ntiles; ++t) {
    auto& v = of_tile[t];
    CHECK((int)v.size() == p.nchunk[t] && !v.empty(), "chunks of tile %d", t);
    std::sort(v.begin(), v.end(), [](const PlanI4& a, const PlanI4& b) { return a.y < b.y; });
    CHECK(v.front().y == p.list_off[t] && v.back().z == p.list_off[t + 1], "tile %d chunk cover", t);
    for (size_t k = 0; k < v.size(); ++k) {
      if (k > 0) CHECK(v[k - 1].z == v[k].y, "tile %d chunks contiguous", t);
      if (v.size() == 1) CHECK(v[k].w == -1 && p.slot0[t] == -1, "single-chunk tile %d slot", t);
      else CHECK(v[k].w == p.slot0[t] + (int)k, "tile %d slot of chunk %zu", t, k);
    }
    if (v.size() > 1) slots += (int)v.size();
  }
  CHECK(slots == p.nslots, "slots");

  // the stored walk, and its meaning: per chunk, sum each item's 2 x 2
  // contribution; per tile, add the chunks; compare with the scatter of every
  // visibility's footprint.  Kernel weights and values are random per
  // visibility (the check is about structure, not about the kernel).
  std::vector<double> wr(M * J), wc(M * J), vr(M), vi(M);
  for (auto& x : wr) x = unif(rng);
  for (auto& x : wc) x = unif(rng);
  for (int64_t i = 0; i < M; ++i) vr[i] = unif(rng), vi[i] = unif(rng);
  std::vector<double> scat(2 * (size_t)L * L, 0.0), gath(2 * (size_t)L * L, 0.0);
  for (int64_t i = 0; i < M; ++i)
    for (int a = 0; a < J; ++a)
      for (int b = 0; b < J; ++b) {
        const size_t cidx = (size_t)((k0[2 * i] + a) % L) * L + (k0[2 * i + 1] + b) % L;
        const double w = wr[i * J + a] * wc[i * J + b];
        scat[2 * cidx] += w * vr[i];
        scat[2 * cidx + 1] += w * vi[i];
      }
  CHECK((int)p.item_row.size() == nchunks && (int)p.tab.size() == nchunks * prm.tab_stride, "table sizes");
  int64_t rows = 0;
  const int HB = T / 2;
  for (int q = 0; q < nchunks; ++q) {
    const PlanI4 ch = p.chunks[q];
    const uint16_t* P = p.tab.data() + (size_t)q * prm.tab_stride;
    const int Wt = P[NO];
    CHECK(P[0] == 0, "chunk %d prefix start", q);
    CHECK(p.item_row[q] == rows, "chunk %d item rows", q);
    rows += (Wt + NT - 1) / NT;
    const int R0 = (ch.x / TD) * T, C0 = (ch.x % TD) * T;
    std::vector<int> per_owner(NO, 0);
    int last_o = -1, last_kr = -1;
    for (int j = 0; j < NT; ++j) {
      const int t0 = (int)(((int64_t)j * Wt + NT - 1) / NT), t1 = (int)(((int64_t)(j + 1) * Wt + NT - 1) / NT);
      for (int s = 0; s < t1 - t0; ++s) {
        const uint32_t it = p.items[(size_t)(p.item_row[q] + s) * NT + j];
        const int e = (int)(it & ((1u << kItemEntryBits) - 1)), ar = (int)((it >> 12) & 15u);
        const int bc = (int)((it >> 16) & 15u), o = (int)(it >> 20);
        CHECK(e < ch.z - ch.y && o < NO && ar <= J && bc <= J, "chunk %d item fields", q);
        const int R = 2 * (o / HB), C = 2 * (o % HB);
        const int key = p.lkey[ch.y + e], kr = key / W, kc = key % W;
        CHECK(ar == R + J - kr && bc == C + J - kc, "chunk %d item taps", q);
        // owners in order, and within an owner the start rows in order
        CHECK(o > last_o || (o == last_o && kr >= last_kr), "chunk %d walk order", q);
        last_o = o;
        last_kr = kr;
        per_owner[o]++;
        const int i = p.perm[p.list[ch.y + e]];
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            const int ta = ar + a - 1, tb = bc + b - 1;  // unpadded taps
            if (ta < 0 || ta >= J || tb < 0 || tb >= J) continue;
            const size_t cidx = (size_t)(R0 + R + a) * L + (C0 + C + b);
            const double w = wr[i * J + ta] * wc[i * J + tb];
            gath[2 * cidx] += w * vr[i];
            gath[2 * cidx + 1] += w * vi[i];
          }
      }
    }
    for (int o = 0; o < NO; ++o) CHECK(P[o + 1] - P[o] == per_owner[o], "chunk %d owner %d work", q, o);
  }
  CHECK(rows == p.nitem_rows && p.items.size() == (size_t)rows * NT, "item rows");
  double err = 0.0, ref = 0.0;
  for (size_t k = 0; k < scat.size(); ++k) {
    err = std::max(err, std::fabs(gath[k] - scat[k]));
    ref = std::max(ref, std::fabs(scat[k]));
  }
  CHECK(err <= 1e-12 * std::max(1.0, ref), "gather vs scatter: max error %.3e (max %.3e)", err, ref);

  // degridding units: each tile's home run in contiguous pieces
  std::vector<int64_t> covered(ntiles, 0);
  for (const PlanI4& d : p.dchunks) {
    CHECK(d.x >= 0 && d.x < ntiles && d.y >= p.home[d.x] && d.z <= p.home[d.x + 1] && d.z > d.y, "degrid unit");
    covered[d.x] += d.z - d.y;
  }
  for (int t = 0; t < ntiles; ++t) CHECK(covered[t] == p.home[t + 1] - p.home[t], "degrid cover of tile %d", t);
  CHECK((int64_t)p.dchunks.size() <= prm.max_partials, "degrid units");
  std::printf("ok chunks=%d multi_slots=%d items=%lld\n", nchunks, p.nslots, (long long)(rows * NT));
  return 0;
}
