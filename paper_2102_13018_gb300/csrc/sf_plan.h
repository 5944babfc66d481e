// sf_plan.h -- index plans built by the setup pass (Sec. V.A-B) and read by the kernels.
//
// Two plans describe the same edges:
//  * the two-sided plan ("TS"): edges grouped by (root rank p, leaf rank q) with q == p first
//    (Sec. V.B: self moved to the head), canonical order inside a group, cut into runs.  A run
//    iterates k = i + nx*(j + ny*z); a side without index array addresses unit
//    base + i + j*sy + z*sz (the multi-strided sub-block start+X*Y*k+X*j+i of Sec. V.B, with
//    contiguous runs as the 1-D case); an indexed side reads idx[idx0 + k].
//  * the root-major plan ("RM"): roots with exactly one leaf as masked contiguous runs or as
//    explicit pairs; roots with several leaves in CSR form (leaves in canonical order), cut
//    into blocks of FOLD_BLOCK leaves for the deterministic fold.
#pragma once
#include <cstdint>

namespace sfgb {

constexpr int FOLD_BLOCK = 64;        // block of the fold D (SF_FOLD_BLOCK)
constexpr int TS_TILE_EDGES = 4096;   // edges per tile of a TS run
constexpr int RM_TILE_EDGES = 4096;   // edges per masked / pairs tile
constexpr int RM_TILE_CHUNKS = 1024;  // fold blocks per chunk tile (at most)
constexpr int RM_TILE_CHUNK_EDGES = 8192;   // leaves per chunk tile (at most)
constexpr int RM_TILE_ROOTS = 1024;   // multi roots per winner tile
constexpr int RM_TILE_FETCH = 128;    // multi roots per fetch tile

enum RunFlags : int32_t {
  RUN_ROOT_IDX = 1,    // root side indexed
  RUN_LEAF_IDX = 2,    // leaf side indexed
  RUN_SELF = 4,        // root rank == leaf rank
  RUN_DUP = 8,         // some root of the run has in-degree > 1 (Reduce must use atomics)
};

struct Run {
  int64_t root0, rsy, rsz;   // root pattern
  int64_t leaf0, lsy, lsz;   // leaf pattern
  int64_t idx0;              // first entry of this run in the TS index arrays
  int64_t rbuf0;             // offset (units) in the root-side buffer (remote runs)
  int64_t lbuf0;             // offset (units) in the leaf-side buffer (remote runs)
  int32_t n, nx, ny, flags;
};

struct Tile {
  int32_t kind;   // TileKind
  int32_t a;      // run / first pair / first chunk / first multi root
  int32_t k0;     // first edge inside the run (TS, masked)
  int32_t cnt;    // number of edges / pairs / chunks / roots
};

enum TileKind : int32_t {
  T_RUN = 0,       // TS run slice
  T_MASKED = 1,    // RM masked run slice
  T_PAIRS = 2,     // RM explicit single-leaf roots
  T_CHUNKS = 3,    // RM fold blocks of multi roots
  T_WINNERS = 4,   // RM multi roots, last leaf in canonical order
  T_FETCH = 5,     // RM multi roots, serial fetch-and-op
};


// A slice [k0, k0+cnt) of a TS run with the run's description inlined (one 96-byte load,
// prefetched by the kernel while it works on the previous tile).
struct TsTile {
  int64_t root0, rsy, rsz;
  int64_t leaf0, lsy, lsz;
  int64_t idx0, rbuf0, lbuf0;
  int32_t n, nx, ny, flags;
  int32_t k0, cnt;
};
static_assert(sizeof(TsTile) == 96, "TsTile is copied in 16-byte pieces");

// A tile of the root-major plan; masked tiles carry their run inline.
struct RmTile {
  int32_t kind;              // T_MASKED, T_PAIRS, T_CHUNKS, T_WINNERS, T_FETCH
  int32_t a;                 // first pair / block / multi root
  int32_t k0;                // masked: first root of the slice inside the run
  int32_t cnt;               // roots / pairs / blocks in the tile
  int64_t root0, leaf0;      // masked run start
  int64_t mask0;             // masked run's first mask bit
  int64_t pad;
};
static_assert(sizeof(RmTile) == 48, "RmTile is copied in 16-byte pieces");

struct MaskedRun {
  int64_t root0, leaf0, mask0;   // mask0: first bit (multiple of 32) in the mask words
  int32_t n, pad;
};

// One fold block of a multi-leaf root: leaves m_leaf[e0 .. e0+n).
struct Block {
  int32_t root;   // root unit
  int32_t e0;     // first edge of the block in m_leaf
  int32_t n;      // leaves in the block (1..FOLD_BLOCK)
  int32_t comb;   // -1 when the root has one block, else its Comb record
};

// A root with several fold blocks: where its block partials and arrival counter live.
// Blocks are folded in two levels, the way D is defined: the partials of each run of
// FOLD_BLOCK consecutive blocks (a super-block) are folded by the super-block's last arriving
// block, and the super-block results by the last arriving super-block.
struct Comb {
  int32_t slot;     // first level-0 partial slot (one per block)
  int32_t slot1;    // first level-1 partial slot (one per super-block)
  int32_t ctr;      // first counter: one per super-block, then one for the root
  int32_t nch;      // number of blocks
  int32_t e_first;  // first edge of the root in m_leaf
  int32_t root;     // root unit
};

// A fold block as stored: 8 bytes.  who >= 0 is the root unit of a single-block root,
// who < 0 is -(Comb index + 1); the block's leaf count is the next record's e0 minus its own
// (blocks are stored in m_leaf order, with one sentinel record after the last).
struct BlockRec {
  int32_t who;
  int32_t e0;
};

struct SegCopy {                 // one (root rank -> leaf rank) chunk of the buffer move
  int64_t src0, dst0, n;         // units
};

// Device view of every plan array (pointers into one device allocation).
struct DevPlan {
  // TS plan
  const int32_t *ts_ridx, *ts_lidx;
  const TsTile *ts_tiles;        // all runs
  const TsTile *ts_self_tiles;   // self runs only (3-phase: direct scatter)
  const TsTile *ts_remote_tiles; // remote runs only (3-phase: pack / unpack)
  const SegCopy *segs;           // remote segments for the move
  int32_t n_ts_tiles, n_ts_self_tiles, n_ts_remote_tiles, n_segs;
  int64_t remote_units;          // units in each 3-phase buffer
  // RM plan
  const uint32_t *mask;
  const int32_t *pr_root, *pr_leaf;
  const int32_t *m_root, *m_ptr, *m_leaf;   // multi roots: root unit, CSR pointers, leaf units
  const BlockRec *blocks;                   // fold blocks of multi roots (+ sentinel)
  const Comb *combs;                        // multi roots with several blocks
  const RmTile *rm_fold_tiles;              // masked + pairs + chunks
  const RmTile *rm_winner_tiles;            // masked + pairs + winners
  const RmTile *rm_fetch_tiles;             // masked + pairs + fetch
  int32_t n_rm_fold_tiles, n_rm_winner_tiles, n_rm_fetch_tiles;
  int32_t n_multi, n_partial_slots, n_counters;
};

}  // namespace sfgb
