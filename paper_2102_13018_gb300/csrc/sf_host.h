// sf_host.h -- host-side graph copy and plan construction (the setup pass, Sec. V.A-B).
#pragma once
#include <cstdint>
#include <memory>
#include <vector>

#include "sf.h"
#include "sf_plan.h"

namespace sfgb {

// The graph as given to sf_create (Sec. III.A), copied and validated.
struct Graph {
  int32_t P = 0;
  std::vector<int64_t> nroots, nleaves;
  std::vector<uint8_t> has_ilocal;
  std::vector<int64_t> ilocal;   // [E], rank-major; entries of ranks without ilocal unused
  std::vector<int32_t> rrank;    // [E]
  std::vector<int64_t> rindex;   // [E]
  std::vector<int64_t> rootoff, leafoff, edgeoff;  // [P+1]
  int64_t E = 0;
};

// Diagonal chunks of the deterministic Reduce, on the host (sf_plan.h, DiagChunk).
struct DiagHost {
  std::vector<DiagChunk> chunks;
  std::vector<int32_t> x, lists;
  std::vector<DgTile> tiles;
  int64_t c0 = 0;
  int64_t roots = 0, extras = 0, list_roots = 0;
};

// Every plan array on the host, before upload.
struct HostPlan {
  std::vector<Run> runs;
  std::vector<int32_t> ts_ridx, ts_lidx;
  std::vector<TsTile> ts_tiles, ts_self_tiles, ts_remote_tiles;
  std::vector<SegCopy> segs;
  int64_t remote_units = 0;

  std::vector<MaskedRun> mruns;
  std::vector<uint32_t> mask;
  std::vector<int32_t> pr_root, pr_leaf;
  std::vector<int32_t> m_root, m_ptr, m_leaf;
  std::vector<Block> blocks;         // host view (tiling, statistics)
  std::vector<BlockRec> block_recs;  // device form, one sentinel record at the end
  std::vector<Comb> combs;
  std::vector<RmTile> rm_fold_tiles, rm_fold_nv1_tiles, rm_winner_tiles, rm_fetch_tiles;
  int32_t n_partial_slots = 0, n_counters = 0;

  std::vector<int32_t> z_root;      // roots without leaves (zeroed by the operations from zero)
  DiagHost dg;                      // diagonal chunks (empty: none)
  std::shared_ptr<HostPlan> rest;   // root-major plan of the roots the diagonal chunks leave out
};

// Validate and copy the arguments of sf_create.  Returns an SF_* code.
int build_graph(int32_t nranks, const int64_t nroots[], const int64_t nleaves[],
                const int64_t *const ilocal[], const sf_node *const iremote[], Graph &g);

// Same, with each rank's leaf extent given (at least max(ilocal)+1): a derived forest keeps the
// buffer layout of the forest it came from.
int build_graph_extents(int32_t nranks, const int64_t nroots[], const int64_t nleaves[],
                        const int64_t *const ilocal[], const sf_node *const iremote[], const int64_t extents[],
                        Graph &g);

// The setup pass: two-sided grouping, pattern detection, root-major plan, statistics.
int analyze(const Graph &g, HostPlan &plan, sf_info &info);

// The two-sided tiles of every run of the plan, `per` edges each (sf_set_tile_edges).
void cut_ts_tiles(const HostPlan &plan, int32_t per, std::vector<TsTile> &out);

}  // namespace sfgb
