/* sf.h -- C ABI of libsfgb, star-forest communication on one GB300 GPU.
 *
 * A star forest (Sec. III.A) is a set of disjoint stars: each root has zero or more leaves,
 * each leaf at most one root.  The graph is described per simulated rank p by the owner of
 * the leaves: nroots[p] roots, nleaves[p] connected leaves with local indices ilocal[p]
 * (NULL = 0..nleaves[p]-1) and their root addresses iremote[p][i] = (rank, index).
 * All ranks live in one GPU's memory.  Their data sits back to back, rank-major:
 *   rootdata unit rootoff[p] + r  is root r of rank p,   rootoff[p] = sum_{p'<p} nroots[p']
 *   leafdata unit leafoff[q] + l  is leaf l of rank q,   leafoff[q] = sum_{q'<q} extent[q']
 * where a rank's leaf extent is max(ilocal[q])+1, or nleaves[q] when ilocal[q] is NULL.
 * A unit is bs consecutive elements of one dtype (the MPI datatype "unit" of Sec. III.B).
 * Edge e = (q, i) is the i-th leaf rank q describes; canonical edge order is ascending (q, i).
 *
 * Conventions shared by every call:
 *  - Every call returns an int error code, SF_SUCCESS (0) on success (Sec. III.A: all
 *    PetscSF routines return an error code).  Nothing aborts or throws across the ABI.
 *  - Graph arrays are copied by sf_create and stay owned by the caller.
 *  - rootdata / leafdata / leafupdate are device pointers owned by the caller, except in the
 *    *_with_memtype calls.  They must be aligned to the element size of the unit's dtype.
 *  - sf_stream_t is a cudaStream_t passed as void*; NULL is the legacy default stream.
 *    Every operation is enqueued on that stream in order, with no host synchronisation.
 *    Results are valid on that stream after the matching End (Sec. III.B: begin/end take
 *    the same arguments; buffers must not change between them).
 *  - Leaves not listed in ilocal and roots without leaves are never written.
 *  - Calls on one sf_t are not thread safe; different sf_t may be used concurrently.
 */
#ifndef SFGB_SF_H
#define SFGB_SF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sf_s sf_t;
typedef struct sf_batch_s sf_batch_t;
typedef void *sf_stream_t;

/* Root address of a leaf: PetscSFNode {rank, offset} of Sec. III.A. */
typedef struct {
  int32_t rank;
  int64_t index;
} sf_node;

/* Element types of a unit. */
enum { SF_INT32 = 0, SF_INT64 = 1, SF_FP32 = 2, SF_FP64 = 3, SF_BF16 = 4 };

/* A unit: bs consecutive elements of dtype, 1 <= bs and bs x element size <= SF_MAX_UNIT_BYTES
 * (larger units are rejected with SF_ERR_ARG; the kernels index a tile's work in 32 bits). */
#define SF_MAX_UNIT_BYTES (1 << 19)
typedef struct {
  int32_t dtype;
  int32_t bs;
} sf_unit;

/* Reduction operators of Sec. III.B (MPI_REPLACE, MPI_SUM, MPI_MIN, MPI_MAX).
 * op(a, b) with a the current value and b the incoming one: REPLACE b, SUM a + b (integers
 * wrap around), MIN (b < a ? b : a), MAX (a < b ? b : a).  On a tie MIN/MAX keep the current
 * value, so equal floating values with different bits (+0 and -0) resolve by the order the
 * operation applies them (canonical edge order in SF_MODE_DETERMINISTIC).  Floating MIN/MAX of
 * NaN input is undefined: the deterministic fold may let a NaN leaf hide the leaves after it. */
enum { SF_REPLACE = 0, SF_SUM = 1, SF_MIN = 2, SF_MAX = 3 };

/* How Reduce combines several leaves of one root (Sec. V.C uses atomics on duplicates).
 * DETERMINISTIC: each root combines its leaves in canonical edge order; a floating point SUM
 *   adds the blocked left fold D of the leaf values (block SF_FOLD_BLOCK, see below) to the
 *   root; bit-identical from run to run.
 * ATOMIC: device atomics in whatever order the hardware applies them.
 * AUTO: the library picks (currently DETERMINISTIC, or what sf_autotune measured fastest).
 * Reduce REPLACE always takes the value of the root's last leaf in canonical order;
 * bf16 SUM always accumulates in fp32 deterministically and rounds once. */
enum { SF_MODE_AUTO = 0, SF_MODE_ATOMIC = 1, SF_MODE_DETERMINISTIC = 2 };

/* Blocked fold D(y_0..y_{n-1}): if n <= SF_FOLD_BLOCK, ((y_0 + y_1) + ...) + y_{n-1};
 * otherwise D of the list of left folds of consecutive blocks of SF_FOLD_BLOCK values. */
#define SF_FOLD_BLOCK 64

/* Data paths for Bcast (Sec. V.B):
 * FUSED: one scatter kernel per operation, leafdata[leaf] op= rootdata[root] for every edge,
 *   grouped by (root rank, leaf rank) with self first; index-free on detected patterns.
 * THREE_PHASE: pack remote edges into a root buffer, move each (root rank -> leaf rank) chunk
 *   into a leaf buffer, unpack into leafdata; self edges are scattered directly.
 * ROOT_MAJOR: each root unit is read once and written to all of its leaves.
 * AUTO: what sf_autotune measured fastest, else ROOT_MAJOR for units of 64 bytes or more on
 *   forests with at least 4 leaves per connected root on average, else FUSED. */
enum { SF_PATH_AUTO = 0, SF_PATH_FUSED = 1, SF_PATH_THREE_PHASE = 2, SF_PATH_ROOT_MAJOR = 3 };

/* Plans of the deterministic Reduce of one-vector units (SUM/MIN/MAX; results are identical):
 * ROOT_MAJOR: CSR-by-root fold tiles with a two-level combine for roots that span tiles.
 * DIAGONAL: 32-root chunks whose roots each own a leaf at one common offset from the root
 *   (Sec. V.B's contiguous patterns, per chunk), then the root-major plan of the roots left
 *   out; only on forests where the setup pass found such chunks (sf_info.dg_chunks > 0).
 * DIAGONAL_STAGED: DIAGONAL with each tile's spans staged in shared memory by bulk copies
 *   (a single forest's Reduce; in a batch it runs as DIAGONAL).
 * AUTO: ROOT_MAJOR, or what sf_autotune measured fastest. */
enum { SF_PLAN_AUTO = 0, SF_PLAN_ROOT_MAJOR = 1, SF_PLAN_DIAGONAL = 2, SF_PLAN_DIAGONAL_STAGED = 3 };

/* Where data lives, for the *_with_memtype calls (PetscSFBcastWithMemTypeBegin, Sec. V.C). */
enum { SF_MEM_HOST = 0, SF_MEM_DEVICE = 1 };

/* Error codes. */
enum {
  SF_SUCCESS = 0,
  SF_ERR_ARG = 1,          /* invalid argument (size, dtype, bs, op, mode, memtype) */
  SF_ERR_NULL = 2,         /* required pointer is NULL */
  SF_ERR_RANGE = 3,        /* iremote rank/index or ilocal out of range */
  SF_ERR_DUP_LEAF = 4,     /* a rank lists the same local leaf twice (stars must be disjoint) */
  SF_ERR_STATE = 5,        /* call out of order (e.g. operation before sf_setup) */
  SF_ERR_NO_PENDING = 6,   /* End without a matching Begin */
  SF_ERR_PENDING = 7,      /* Begin already pending with these arguments, or destroy with one */
  SF_ERR_UNSUPPORTED = 8,  /* valid but not supported (e.g. atomic FetchAndOp with bs > 1) */
  SF_ERR_ALLOC = 9,        /* host or device allocation failed */
  SF_ERR_CUDA = 10,        /* a CUDA runtime call failed (no device, launch failure, ...) */
  SF_ERR_ALIGN = 11,       /* data pointer not aligned to the element size */
  SF_ERR_TOO_LARGE = 12    /* sizes beyond what the library indexes (2^31-1 units) */
};

/* Statistics of the setup pass (Sec. V.A-B), valid after sf_analyze or sf_setup. */
typedef struct {
  int32_t nranks;
  int32_t analyzed;
  int32_t setup_done;
  int32_t has_dup_roots;       /* some root has in-degree > 1 (Sec. V.C) */
  int64_t nroots_total;        /* rootoff[nranks] */
  int64_t leaf_extent_total;   /* leafoff[nranks] */
  int64_t nedges;
  int64_t max_in_degree;
  int64_t connected_roots;     /* roots with in-degree >= 1 */
  int64_t multi_roots;         /* roots with in-degree >= 2 */
  int64_t multi_edges;         /* edges into those roots */
  int64_t segments;            /* non-empty (root rank, leaf rank) pairs */
  int64_t self_edges;          /* edges whose root and leaf rank agree */
  int64_t runs;                /* runs of the (root rank, leaf rank) edge order */
  int64_t runs_pattern;        /* runs with both sides index-free (contiguous / 3-D) */
  int64_t runs_3d;             /* of those, with more than one row */
  int64_t edges_both_pattern;  /* edges with no index load on either side */
  int64_t edges_one_indexed;   /* edges with exactly one side index-driven */
  int64_t edges_two_indexed;   /* edges with both sides index-driven */
  int64_t rm_masked_runs;      /* root-major plan: contiguous single-leaf runs */
  int64_t rm_masked_edges;
  int64_t rm_pairs;            /* root-major plan: other single-leaf roots */
  int64_t rm_chunks;           /* root-major plan: blocks of SF_FOLD_BLOCK leaves of multi roots */
  int64_t device_plan_bytes;   /* device memory held by the plans */
  int64_t ts_tile_edges;       /* edges per tile of a two-sided run (smaller forests: smaller tiles) */
  int64_t rm_tile_edges;       /* edges per masked / single-leaf tile of the root-major plan */
  int64_t rm_tile_blocks;      /* fold blocks per chunk tile of the root-major plan (at most) */
  int64_t dg_chunks;           /* diagonal-chunk plan of the deterministic Reduce: 32-root chunks (0: none) */
  int64_t dg_roots;            /* roots it covers (each with its leaf at root + a per-chunk offset) */
  int64_t dg_extra_leaves;     /* their other leaves */
  int64_t dg_list_roots;       /* of those roots, with more than one other leaf */
  int64_t dg_rest_roots;       /* connected roots it leaves to the root-major plan */
} sf_info;

/* Create a star forest (PetscSFCreate + PetscSFSetGraph, Sec. III.A).
 * nranks >= 1; nroots[p], nleaves[p] >= 0; ilocal may be NULL (all ranks contiguous) and
 * ilocal[p] may be NULL; iremote[p] may be NULL only when nleaves[p] == 0.  The arrays are
 * validated (ranges, duplicate leaves) and copied.  *out receives the handle.
 * Errors: SF_ERR_NULL, SF_ERR_ARG, SF_ERR_RANGE, SF_ERR_DUP_LEAF, SF_ERR_TOO_LARGE, SF_ERR_ALLOC. */
int sf_create(int32_t nranks, const int64_t nroots[], const int64_t nleaves[],
              const int64_t *const ilocal[], const sf_node *const iremote[], sf_t **out);

/* Host part of PetscSFSetUp (Sec. V.A-B): two-sided grouping by (root rank, leaf rank) with
 * self first, pattern detection (contiguous and multi-strided 3-D runs), duplicate-root
 * detection, root-major plan.  Needs no GPU.  Idempotent. */
int sf_analyze(sf_t *sf);

/* PetscSFSetUp (Sec. III.A): sf_analyze if not done, then upload the plans to the current
 * CUDA device and allocate the persistent buffers.  Enqueued on `stream`; synchronises it
 * once before returning.  Errors: SF_ERR_CUDA, SF_ERR_ALLOC. */
int sf_setup(sf_t *sf, sf_stream_t stream);

/* rootoff[nranks+1] and leafoff[nranks+1] of the concatenated buffers (caller-allocated). */
int sf_get_layout(const sf_t *sf, int64_t *rootoff, int64_t *leafoff);

int sf_get_info(const sf_t *sf, sf_info *info);

/* Select the Reduce mode (SF_MODE_*) and the Bcast data path (SF_PATH_*). */
int sf_set_mode(sf_t *sf, int32_t mode);
int sf_set_path(sf_t *sf, int32_t path);
/* Select the deterministic Reduce plan (SF_PLAN_*); a forest without diagonal chunks runs
 * ROOT_MAJOR whatever is set. */
int sf_set_reduce_plan(sf_t *sf, int32_t plan);

/* Launch shape of the forest's kernels (the choices sf_autotune makes; results do not change):
 * vector_bytes caps the vector each thread moves per unit access (2, 4, 8 or 16; 0 = 16; a unit's
 * element size is always allowed), and tile_edges sets the edges per CTA tile of the two-sided
 * kernels (fused Bcast, atomic Reduce): a power of two in [64, 65536], 0 = the setup pass's
 * choice (sf_info.ts_tile_edges).  sf_set_tile_edges rebuilds that tile list on the device: it
 * needs sf_setup, allocates, synchronises the device and refuses (SF_ERR_PENDING) while a Begin
 * has no End. */
int sf_set_vector_bytes(sf_t *sf, int32_t bytes);
int sf_set_tile_edges(sf_t *sf, int32_t edges);

typedef struct {
  int32_t path;          /* SF_PATH_* the Bcast runs (AUTO resolved; for units under 64 bytes) */
  int32_t mode;          /* SF_MODE_* the Reduce runs (AUTO resolved) */
  int32_t vector_bytes;  /* 0 = 16 */
  int32_t tile_edges;    /* edges per two-sided tile */
  int32_t reduce_plan;   /* SF_PLAN_* the deterministic Reduce runs (AUTO resolved) */
} sf_tuning;

/* The forest's current choices (after sf_autotune, or as set). */
int sf_get_tuning(const sf_t *sf, sf_tuning *out);

/* Bcast (Sec. III.B): for every edge, leafdata[leaf] = op(leafdata[leaf], rootdata[root]).
 * Begin enqueues the work on `stream` (all of it for FUSED/ROOT_MAJOR; pack, self scatter and
 * move for THREE_PHASE); End enqueues what remains (the unpack) and must repeat the arguments.
 * rootdata must not alias leafdata.  Errors: SF_ERR_STATE, SF_ERR_ARG, SF_ERR_NULL,
 * SF_ERR_ALIGN, SF_ERR_PENDING, SF_ERR_NO_PENDING, SF_ERR_CUDA. */
int sf_bcast_begin(sf_t *sf, sf_unit unit, const void *rootdata, void *leafdata, int32_t op,
                   sf_stream_t stream);
int sf_bcast_end(sf_t *sf, sf_unit unit, const void *rootdata, void *leafdata, int32_t op,
                 sf_stream_t stream);

/* Reduce (Sec. III.B): for every edge, rootdata[root] = op(rootdata[root], leafdata[leaf]),
 * combined per root as the mode says (see SF_MODE_*).  Same begin/end rules as Bcast. */
int sf_reduce_begin(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op,
                    sf_stream_t stream);
int sf_reduce_end(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op,
                  sf_stream_t stream);

/* Reduce into roots that start at zero: the result is what sf_reduce_begin/end compute after
 * rootdata was set to zero (with the forest's mode; roots without leaves end at 0), but the old
 * rootdata is never read, and only the roots without leaves are written twice -- cheaper than a
 * memset of the whole root buffer followed by a Reduce.  The functional form the adjoint of
 * Bcast needs (Sec. IV.A: y = P^T lvec).  Same begin/end rules as sf_reduce_begin/end. */
int sf_reduce_from_zero_begin(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op,
                              sf_stream_t stream);
int sf_reduce_from_zero_end(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op,
                            sf_stream_t stream);

/* Set every root without leaves to 0 (all bs elements), and, when argleaf is not NULL, its bs
 * entries of argleaf (int32[nroots_total * bs]) to -1; other roots are not touched.  Together
 * with sf_reduce_maxloc this gives the functional MAX with location over every root. */
int sf_zero_leafless_roots(sf_t *sf, sf_unit unit, void *rootdata, int32_t *argleaf, sf_stream_t stream);

/* FetchAndOp (Sec. III.B): for each root, its leaves are applied one at a time; before leaf
 * e is applied, the root's current value is stored into leafupdate[leaf e]:
 *   leafupdate[leaf] = rootdata[root];  rootdata[root] = op(rootdata[root], leafdata[leaf]).
 * DETERMINISTIC (and AUTO) mode applies a root's leaves in canonical edge order; ATOMIC mode
 * in hardware order (bs must be 1, else SF_ERR_UNSUPPORTED).  leafupdate must not alias
 * leafdata or rootdata. */
int sf_fetch_and_op_begin(sf_t *sf, sf_unit unit, void *rootdata, const void *leafdata,
                          void *leafupdate, int32_t op, sf_stream_t stream);
int sf_fetch_and_op_end(sf_t *sf, sf_unit unit, void *rootdata, const void *leafdata,
                        void *leafupdate, int32_t op, sf_stream_t stream);

/* Bcast/Reduce with explicit memory types (PetscSFBcastWithMemTypeBegin, Sec. V.C):
 * rootmtype / leafmtype are SF_MEM_HOST or SF_MEM_DEVICE.  Host buffers are staged through
 * library-owned device buffers: inputs are copied host->device at Begin, the output is
 * copied device->host at End, all on `stream`.  Host memory should be page-locked for the
 * copies to be asynchronous; pageable memory works but the copies then block the host.
 * The host output is valid once `stream` has completed after End. */
int sf_bcast_with_memtype_begin(sf_t *sf, sf_unit unit, int32_t rootmtype, const void *rootdata,
                                int32_t leafmtype, void *leafdata, int32_t op, sf_stream_t stream);
int sf_bcast_with_memtype_end(sf_t *sf, sf_unit unit, int32_t rootmtype, const void *rootdata,
                              int32_t leafmtype, void *leafdata, int32_t op, sf_stream_t stream);
int sf_reduce_with_memtype_begin(sf_t *sf, sf_unit unit, int32_t leafmtype, const void *leafdata,
                                 int32_t rootmtype, void *rootdata, int32_t op, sf_stream_t stream);
int sf_reduce_with_memtype_end(sf_t *sf, sf_unit unit, int32_t leafmtype, const void *leafdata,
                               int32_t rootmtype, void *rootdata, int32_t op, sf_stream_t stream);

/* ---- Forests derived from a forest (Sec. III.B-C) ----
 * Embedded forests (PetscSFCreateEmbeddedRootSF / LeafSF): only the edges of the selected
 * roots (global root units, i.e. rootoff[p] + r) or selected leaves (global leaf units), with
 * nothing renumbered: the new forest has the same ranks, roots and leaf layout, so the
 * original rootdata / leafdata buffers serve it.  *out is a new forest (set it up before use;
 * destroy it with sf_destroy).  Errors: SF_ERR_NULL, SF_ERR_ARG, SF_ERR_RANGE, SF_ERR_ALLOC. */
int sf_create_embedded_root_sf(const sf_t *sf, int64_t n, const int64_t selected_roots[], sf_t **out);
int sf_create_embedded_leaf_sf(const sf_t *sf, int64_t n, const int64_t selected_leaves[], sf_t **out);

/* Composition (PetscSFCompose): A's leaf space is B's root space (leafoff of A equals rootoff
 * of B rank by rank).  AB has A's roots and B's leaves; B's leaf l connects to A's root a when
 * l's root in B is a leaf of A connected to a (a B leaf whose B root is an isolated A leaf is
 * left out).  Bcast over AB equals Bcast over A then Bcast over B.  New forest in *AB. */
int sf_compose(const sf_t *A, const sf_t *B, sf_t **AB);

/* Inverse composition (PetscSFComposeInverse): A and B share the leaf space, and every root of
 * B has at most one leaf (else SF_ERR_ARG).  AB has A's roots, and B's roots are its leaves: B's
 * root r connects to A's root a when r's leaf is a leaf of A connected to a.  The leaf space of
 * AB is B's root space.  New forest in *AB. */
int sf_compose_inverse(const sf_t *A, const sf_t *B, sf_t **AB);

/* Multi-forest (PetscSFGetMultiSF): every root of degree d becomes d roots, and the k-th leaf of
 * a root in canonical order connects to its k-th new root.  Built on first use with the
 * paper's recipe -- Reduce SUM of ones for the degrees, roots set to their rank's degree prefix
 * sums, FetchAndOp SUM with leaves of 1, each leaf fetching its new root's offset -- which
 * allocates and synchronises `stream`.  *multi is owned by sf (valid until sf_destroy; do not
 * destroy it).  Rank p of the multi-forest owns sum of its roots' degrees roots. */
int sf_get_multi_sf(sf_t *sf, sf_stream_t stream, sf_t **multi);

/* Gather (PetscSFGatherBegin/End): multirootdata[k-th new root of r] = leafdata[k-th leaf of r]
 * (multirootdata has the multi-forest's root layout).  Scatter reverses it.  Both are
 * Reduce / Bcast REPLACE over the multi-forest, with the same begin/end rules. */
int sf_gather_begin(sf_t *sf, sf_unit unit, const void *leafdata, void *multirootdata, sf_stream_t stream);
int sf_gather_end(sf_t *sf, sf_unit unit, const void *leafdata, void *multirootdata, sf_stream_t stream);
int sf_scatter_begin(sf_t *sf, sf_unit unit, const void *multirootdata, void *leafdata, sf_stream_t stream);
int sf_scatter_end(sf_t *sf, sf_unit unit, const void *multirootdata, void *leafdata, sf_stream_t stream);

/* Reduce MAX with location, for the gradient of Reduce MAX.  For every root with leaves,
 * rootdata = the maximum over its leaves (the old root value takes no part) and argleaf = the
 * leaf unit (index into leafdata's units) of the first leaf in canonical order that reaches it,
 * per component; argleaf is int32[nroots_total * bs].  Roots without leaves are not written
 * (initialise rootdata and argleaf, e.g. to 0 and -1).  No NaN in leafdata. */
int sf_reduce_maxloc(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t *argleaf,
                     sf_stream_t stream);

/* Gradient of sf_reduce_maxloc: leafgrad[argleaf[i]*bs + c] = rootgrad[i] for every root
 * element i = r*bs + c with argleaf[i] >= 0; other leaf elements are not written. */
int sf_maxloc_scatter(sf_t *sf, sf_unit unit, const int32_t *argleaf, const void *rootgrad, void *leafgrad,
                      sf_stream_t stream);

/* The same gradient written whole: every connected leaf l of root r gets, per element c,
 * leafgrad[l*bs + c] = rootgrad[r*bs + c] if argleaf[r*bs + c] == l, else 0 (argleaf as
 * sf_reduce_maxloc wrote it).  Leaves with no root are not written, so a forest whose leaves
 * are all connected needs no zero fill of leafgrad first.  Root-major: each leaf unit is
 * written once, no leaf is read.  Same errors as sf_maxloc_scatter. */
int sf_maxloc_grad(sf_t *sf, sf_unit unit, const int32_t *argleaf, const void *rootgrad, void *leafgrad,
                   sf_stream_t stream);

/* ---- Batched execution (Sec. V.D: launch cost and pipelining; CUDA graphs as future work) ----
 * A batch runs many forests' operations with few kernel launches: operations are grouped by
 * kernel variant (element type, op, vector width, data path, Reduce mode) and each group is one
 * launch over all of its operations' tiles.  SF_OP_BARRIER entries split the list into stages
 * that run in order; operations inside a stage run in no particular order and must not write
 * memory that another operation of the same stage reads or writes (and a forest may appear in
 * only one Reduce of a stage).  Each operation uses its forest's current path and mode; the
 * three-phase path runs as the fused path inside a batch. */
enum { SF_OP_BCAST = 0, SF_OP_REDUCE = 1, SF_OP_BARRIER = 2 };

typedef struct {
  sf_t *sf;        /* a set-up forest (ignored for SF_OP_BARRIER) */
  int32_t kind;    /* SF_OP_BCAST, SF_OP_REDUCE or SF_OP_BARRIER */
  sf_unit unit;
  int32_t op;      /* SF_REPLACE .. SF_MAX */
  const void *src; /* Bcast: rootdata; Reduce: leafdata (device memory) */
  void *dst;       /* Bcast: leafdata; Reduce: rootdata (device memory) */
} sf_batch_op;

int sf_batch_create(sf_batch_t **out);

/* Run ops[0..n) on `stream`.  The first call with a given list (or after a forest's path or
 * mode changed) builds and uploads the batch's tables, which allocates device memory and
 * synchronises `stream`; later calls with the same list only launch.  With use_graph != 0 the
 * launches are captured once into a CUDA graph (on a private stream) and every call replays it
 * with one cudaGraphLaunch on `stream`.  Errors: those of the single operations. */
int sf_batch_run(sf_batch_t *batch, const sf_batch_op ops[], int32_t n, int32_t use_graph, sf_stream_t stream);

/* Kernel launches one run of the current list takes (its number of variant groups). */
int sf_batch_launches(const sf_batch_t *batch, int32_t *launches);
int sf_batch_destroy(sf_batch_t *batch);

/* Autotuner: times the variants of Bcast (kind SF_OP_BCAST: data path x vector width x
 * two-sided tile size) or of Reduce (kind SF_OP_REDUCE: mode x vector width, the plan for the
 * deterministic mode and the tile size for the atomic mode) on this forest, unit and op,
 * `reps` times after one warm-up, writing into a scratch copy of dst (src and dst are not
 * modified), and keeps the fastest: its path or mode becomes what SF_PATH_AUTO / SF_MODE_AUTO
 * mean for the forest, a tuned plan what SF_PLAN_AUTO means (when the forest's plan is AUTO),
 * and its vector width and tile size are set (sf_set_vector_bytes, sf_set_tile_edges).
 * *choice (may be NULL) receives the path or mode; sf_get_tuning gives the rest.  Allocates
 * and synchronises.  Choosing SF_MODE_ATOMIC trades bit-reproducibility for speed; pass
 * SF_MODE_DETERMINISTIC as the forest's mode before tuning, and the Reduce keeps it (then only
 * the plan and the vector width are tuned). */
int sf_autotune(sf_t *sf, sf_unit unit, int32_t kind, const void *src, void *dst, int32_t op, int32_t reps,
                sf_stream_t stream, int32_t *choice);

/* Maximum scratch, in bytes, that sf_reduce_noalloc may use (a fixed device array). */
#define SF_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Deterministic Reduce that allocates nothing.  The paper has no counterpart: this exists for
 * callers that may not allocate device memory at the time of the call -- for example an
 * application that hands out all device memory from its own pool under a budget fixed at
 * start-up (a cudaMalloc here would bypass its accounting or fail against its cap), or code
 * running inside a custom allocator's callback, where a nested cudaMalloc could re-enter that
 * allocator.  sf_reduce_begin/end may grow the
 * forest's fold scratch with cudaMalloc on the first operation with a wider unit; this call
 * instead keeps the fold partials and arrival counters in one file-scope device array of
 * SF_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds until exit.
 *
 * Computes exactly what sf_reduce_begin + sf_reduce_end compute in SF_MODE_DETERMINISTIC
 * (bit-identical results), whatever mode the forest is set to, and completes in one call
 * (no End; nothing is left pending).  The forest must be set up (sf_setup); the caller
 * passes leafdata and rootdata as for sf_reduce_begin.
 * The first call on a device looks up the array's device address with cudaGetSymbolAddress
 * (with that device current); make that first call before any stream capture.  Each call
 * clears the counters it uses on `stream` before its kernel.  All calls share the one array:
 * calls whose work overlaps on the GPU (different streams, or concurrent processes' threads
 * on one context) race and give wrong results; serialise them.
 * Errors: those of sf_reduce_begin, and SF_ERR_TOO_LARGE when the forest's fold scratch for
 * this unit exceeds SF_NOALLOC_SCRATCH_BYTES (nothing is launched then). */
int sf_reduce_noalloc(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op,
                      sf_stream_t stream);

/* Free the forest and its device plans.  SF_ERR_PENDING (and nothing freed) if a Begin has
 * no End yet.  Synchronises the device work the library enqueued before freeing. */
int sf_destroy(sf_t *sf);

/* Device status bits of a forest: waits inside the kernels are bounded (about one second);
 * one that runs out sets its bit, skips its tile and lets the kernel finish.  A kernel also
 * checks that each tile it stages fits its shared memory, and skips (with a bit) one that does
 * not -- a plan read by the wrong kernel form, never expected. */
#define SF_DEVSTAT_STAGE_TIMEOUT 1   /* a bulk copy of plan indices into shared memory did not land */
#define SF_DEVSTAT_TILE_REFUSED 2    /* a tile larger than the kernel's shared-memory stage was skipped */

/* The forest's device status bits raised since the previous call (0: none), then cleared.
 * Synchronises `stream` (the work the library enqueued on it).  A nonzero status means the
 * results of the operations since the previous call are not to be trusted.
 * Errors: SF_ERR_NULL, SF_ERR_STATE (no setup), SF_ERR_CUDA. */
int sf_get_device_status(sf_t *sf, sf_stream_t stream, int32_t *status);

/* Static description of an error code (never NULL). */
const char *sf_error_string(int code);

/* Kernels launched by the library since the process started (all entry points). */
int64_t sf_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SFGB_SF_H */
