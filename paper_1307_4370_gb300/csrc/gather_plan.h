// Host-side plan of the interpolation operator G and its adjoint on the
// 2n x 2n grid (§5 eq. opmodel: G is sparse and fixed by the frequencies, so
// its structure is built once).  Plain C++ (no CUDA), so that the planning
// can be compiled and checked on a host without a GPU.
//
// Input: per visibility the first cell (row, column) of its J x J footprint
// on the L x L grid.  Output:
//   - the visibilities sorted by the T x T grid tile of their first cell
//     (stable), and per tile the run of its "home" visibilities;
//   - per tile, the list of sorted indices whose footprint meets the tile,
//     ordered by the footprint's first cell relative to the tile (key =
//     (dr + J - 1) * W + (dc + J - 1), W = T + J - 1);
//   - the gridding work units ("chunks": a run of one tile's list), with
//     per chunk the prefix of the 2 x 2 cell blocks' ("owners'") gather work
//     and the gather items of each of the kernel's threads (see grid_item);
//   - the degridding work units (runs of one tile's home visibilities).
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#ifdef __CUDACC__
#define PURIFY_HD __host__ __device__
#else
#define PURIFY_HD
#endif

namespace purify {

constexpr int kGridThreads = 256;  // threads of one gridding CTA (one slice each)

// One gather step of the gridding: a 32-bit item with the entry index in the
// chunk (12 bits), the padded row tap of the owner's first cell row (4 bits),
// the padded column tap of its first cell column (4 bits) and the owner
// (10 bits).
constexpr int kItemEntryBits = 12;
PURIFY_HD constexpr uint32_t grid_item(int e, int ar, int bc, int o) {
  return (uint32_t)e | ((uint32_t)ar << 12) | ((uint32_t)bc << 16) | ((uint32_t)o << 20);
}

struct alignas(16) PlanI4 {  // same layout as CUDA's int4
  int x, y, z, w;
};

struct GatherPlanParams {
  int64_t M;             // visibilities
  int L;                 // grid side
  int J;                 // footprint side (<= 8)
  int T;                 // tile side (power of two, divides L, <= 64)
  size_t fixed_bytes;    // shared memory of a gridding CTA without its entries
  size_t entry_bytes;    // shared memory per staged entry
  size_t smem_budget;    // target shared memory of a gridding CTA
  int tab_stride;        // 16-bit values per chunk in the owner-prefix table (>= (T/2)^2 + 1)
  int64_t max_partials;  // bound on degridding chunks (one reduction slot each)
};

struct GatherPlan {
  int ntiles = 0, tiles_1d = 0;
  std::vector<int> perm;        // sorted position -> caller index (M)
  std::vector<int> home;        // ntiles + 1: home visibilities of tile t are sorted [home[t], home[t+1])
  std::vector<int> list_off;    // ntiles + 1: list entries of tile t are [list_off[t], list_off[t+1])
  std::vector<int> list;        // sorted index of each list entry
  std::vector<int> lkey;        // start-cell key of each list entry
  int chunk_max = 0;            // entries per gridding chunk at most
  std::vector<PlanI4> chunks;   // (tile, list begin, list end, first partial-tile slot or -1), heavy first
  std::vector<int> slot0;       // per tile: first slot of a multi-chunk tile, else -1
  std::vector<int> nchunk;      // per tile: chunks
  int nslots = 0;               // partial-tile slots
  std::vector<uint16_t> tab;    // per chunk, tab_stride values: owner-work prefix P[0..NO]
  std::vector<int> item_row;    // per chunk: first row of its items
  std::vector<uint32_t> items;  // rows x kGridThreads: step s of thread j of a chunk at row item_row + s, column j
  int64_t nitem_rows = 0;
  std::vector<PlanI4> dchunks;  // degridding units (tile, sorted begin, sorted end, 0), heavy first
};

// Returns 0, or -1 for invalid parameters, -2 when the tile lists exceed
// 2^31 - 1 entries or a chunk's gather table does not fit its 16-bit /
// bit-field encoding.
int build_gather_plan(const int* k0 /* M x 2: first footprint cell (row, column) in [0, L) */,
                      const GatherPlanParams& prm, GatherPlan& out);

}  // namespace purify
