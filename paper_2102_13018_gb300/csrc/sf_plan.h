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
// Tile sizes are powers of two chosen per forest at setup: a launch should have about
// TILE_TARGET tiles (several waves of 152 SMs x several resident CTAs) so that a small forest
// still keeps enough loads in flight; large forests use the maxima below, small ones go down to
// the minima (two units of work per thread of a 256-thread CTA: 256 was 10% slower on a
// batch of 512 small forests, 1024 slowed the 1.2M-edge halo).
constexpr int64_t TILE_TARGET = 4096;
constexpr int TS_TILE_EDGES = 4096;   // edges per tile of a TS run (at most)
constexpr int TS_TILE_EDGES_MIN = 512;
constexpr int RM_TILE_EDGES = 4096;   // edges per masked / pairs tile (at most)
constexpr int RM_TILE_EDGES_MIN = 512;
constexpr int RM_TILE_CHUNKS = 1024;  // fold blocks per chunk tile (at most)
constexpr int RM_TILE_CHUNKS_MIN = 256;
constexpr int RM_TILE_CHUNK_EDGES = 8192;   // leaves per chunk tile (at most), per 1024 blocks
// The one-vector-unit Reduce kernel (NV1) reads a second list of chunk tiles, cut at half
// the leaves, so that its gather buffer fits beside the stages.
constexpr int RM_TILE_CHUNK_EDGES_NV1 = 4096;
// A Reduce chunk tile stages its block records [a, a + cnt] and leaf entries [k0, e1) in shared
// memory with two bulk copies; the spans, widened to 16-byte boundaries, fit these arrays.
constexpr int RM_STAGE_RECS = RM_TILE_CHUNKS + 4;
constexpr int RM_STAGE_LEAVES = RM_TILE_CHUNK_EDGES + 8;
constexpr int RM_STAGE_LEAVES_NV1 = RM_TILE_CHUNK_EDGES_NV1 + 8;
// Leaf vectors an NV1 chunk tile gathers into shared memory per round (bytes): with its two
// stages the kernel stays within 48 KB of static shared memory, and four CTAs fit one SM.
constexpr int RM_FLAT_BYTES = 22 * 1024;
// Multi-vector units fold the same way (FLAT kernels) with up to this many vectors per unit
// (a CTA of 256 threads holds 2 or 4 (block, vector) items per thread; a round holds whole units).
constexpr int RM_FLAT_MAX_NV = 512;
// Device status bits (sf_get_device_status): a bounded wait that ran out; a chunk tile larger
// than the kernel's stage (a tile list that does not belong to the kernel) that was skipped.
constexpr int32_t DEVSTAT_STAGE_TIMEOUT = 1;
constexpr int32_t DEVSTAT_TILE_REFUSED = 2;
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


// A tile of a TS run with the run inline.  Units, strides and edge offsets are below 2^31 (the
// library's size limit), so the device copy keeps them in 32 bits.
struct TsTile {
  int32_t root0, rsy, rsz;
  int32_t leaf0, lsy, lsz;
  int32_t idx0, rbuf0, lbuf0;
  int32_t n, nx, ny, flags;
  int32_t k0, cnt;
  uint32_t mx, my;   // DivMagic of nx and ny (3-D runs)
  int32_t sx, sy;
  int32_t pad;
};
static_assert(sizeof(TsTile) == 80, "TsTile is copied in 16-byte pieces");

// Division by a run-time invariant d >= 1 for numerators 0 <= n < 2^31 as one multiply and one
// shift (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994,
// Sec. 4): with l = ceil(log2 d) and m = floor(2^(31+l) / d) + 1 (so 2^(31+l) < m d <=
// 2^(31+l) + 2^l, and m < 2^32), floor(n / d) = floor(n m / 2^(31+l)).
struct DivMagic {
  uint32_t m;
  int32_t s;
};
inline DivMagic div_magic(uint32_t d) {
  int l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  return DivMagic{uint32_t(((uint64_t(1) << (31 + l)) / d) + 1), 31 + l};
}

// A tile of the root-major plan; masked tiles carry their run inline.
struct RmTile {
  int32_t kind;              // T_MASKED, T_PAIRS, T_CHUNKS, T_WINNERS, T_FETCH
  int32_t a;                 // first pair / block / multi root
  int32_t k0;                // masked: first root of the slice inside the run; chunks: first leaf entry
  int32_t cnt;               // roots / pairs / blocks in the tile
  int64_t root0, leaf0;      // masked run start
  int64_t mask0;             // masked run's first mask bit
  int64_t e1;                // chunks: one past the last leaf entry (the span is m_leaf[k0, e1))
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

// Diagonal chunks (deterministic Reduce, see build_diag): chunk c covers root units
// 32 (c0 + c) .. + 31, one 2-bit code per root -- DG_SKIP (not in this plan), DG_DIAG (its one
// leaf is the diagonal leaf root + delta), DG_PAIR (the diagonal leaf and one more, whose x
// entry is its leaf unit, top bit set when it comes after the diagonal one in canonical order),
// DG_LIST (its x entry points at a list: header -1 - (leaves before | leaves after << 16), a
// negative number, then the other leaf units in canonical order).  Roots with DG_PAIR or DG_LIST
// take one x entry each,
// in root order from xoff on.
enum : uint32_t { DG_SKIP = 0, DG_DIAG = 1, DG_PAIR = 2, DG_LIST = 3 };
constexpr int32_t DG_MAX_LEAVES = 64;        // one fold block: D is the plain left fold
constexpr int32_t DG_MIN_CHUNK_ROOTS = 8;    // a chunk with fewer diagonal roots is left to the rest
constexpr int64_t DG_MIN_ROOTS = 1024;       // fewer diagonal roots in all: no diagonal plan
struct DiagChunk {
  uint32_t lo, hi;   // codes of roots 0..15 and 16..31 of the chunk
  int32_t xoff;      // first x entry of the chunk
  int32_t delta;     // diagonal leaf unit - root unit
};
static_assert(sizeof(DiagChunk) == 16, "one 16-byte load per chunk");
// A tile of the staged diagonal-chunk kernel: chunks [c, c + n) of the plan (n <= DG_TILE_CHUNKS),
// one delta, x entries [xbeg, xend) (at most DG_TILE_XCAP), list entries [lbeg, lend) (at most
// DG_TILE_LCAP), and whether every root of the tile (below the forest's last root) is in the
// plan.
constexpr int32_t DG_TILE_CHUNKS = 32;
constexpr int32_t DG_TILE_XCAP = 512;   // the SpMV scatter's tiles hold about 154 on average
constexpr int32_t DG_TILE_LCAP = 256;   // and about 6 list roots
struct DgTile {
  int32_t c, n, delta, xbeg, xend, full, lbeg, lend;
};
static_assert(sizeof(DgTile) == 32, "tile descriptors are read as two 16-byte vectors");

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
  const RmTile *rm_fold_nv1_tiles;          // masked + pairs + chunks of at most RM_TILE_CHUNK_EDGES_NV1
  const RmTile *rm_winner_tiles;            // masked + pairs + winners
  const RmTile *rm_fetch_tiles;             // masked + pairs + fetch
  int32_t n_rm_fold_tiles, n_rm_fold_nv1_tiles, n_rm_winner_tiles, n_rm_fetch_tiles;
  int32_t n_multi, n_partial_slots, n_counters;
  // diagonal chunks (deterministic Reduce); the root-major plan of the roots they leave out is a
  // second DevPlan whose root-major arrays alone are set
  const DiagChunk *dg_chunks;
  const int32_t *dg_x, *dg_lists;
  int32_t dg_c0, dg_nchunks;
  const int32_t *z_root;   // roots without leaves
  int32_t n_z_root;
  const DgTile *dg_tiles;  // tiles of the staged diagonal-chunk kernel
  int32_t n_dg_tiles;
};

}  // namespace sfgb
