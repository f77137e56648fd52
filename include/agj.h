/*
 * agj.h — C ABI of the GB300-native adaptive geospatial join (probe side).
 *
 * Method: Kipf et al., "Adaptive Geospatial Joins for Modern Hardware".
 *   §III-A  five phases: build logical index, build physical index, training,
 *           probe, refine; parameters: precision (metres) and memory budget.
 *   §III-B  logical index = "super covering" of coverings and interior
 *           coverings with precision-preserving conflict resolution
 *           (Listing "Build super covering").
 *   §III-C  physical index = Adaptive Cell Trie (256-ary radix tree over cell
 *           ids, tagged 8-byte entries) + lookup table of reference lists.
 *   §III-D  training on historical points.
 *   §III-E  probe (Listings "Probe Adaptive Cell Trie", "The probe algorithm").
 *
 * Conventions for every entry point:
 *   - returns AGJ_OK (0) or a positive AGJ_E* status; agj_strerror() names it;
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are CPU memory (pinned memory makes copies
 *     asynchronous, pageable memory is accepted too);
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); work is enqueued on it and runs asynchronously unless the
 *     entry point says it synchronises;
 *   - points are n x {lat, lng} FP64 degrees, interleaved (16 bytes per point,
 *     16-byte aligned); a point is valid iff both are finite, |lat| <= 90 and
 *     |lng| <= 180; an invalid point joins no polygon (an empty CSR row) and
 *     is not an error;
 *   - polygon ids are input positions 0 .. n_polys-1 (fewer than 2^30 - 1,
 *     §III-C: 30-bit payloads).
 */
#ifndef AGJ_H
#define AGJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------------- */
/* status codes                                                             */
/* ---------------------------------------------------------------------- */
#define AGJ_OK            0
#define AGJ_EINVAL        1   /* null pointer, bad size, malformed polygon, invalid vertex */
#define AGJ_EUNSUPPORTED  2   /* polygon not within one cube face, >= 2^30-1 polygons */
#define AGJ_EBUDGET       3   /* approximate index would exceed the memory budget (§III-A) */
#define AGJ_ENOMEM        4   /* host or device allocation failed */
#define AGJ_ECUDA         5   /* a CUDA runtime call failed */
#define AGJ_ETIMEOUT      6   /* a bounded device wait gave up (device status word) */
#define AGJ_EBUSY         7   /* server admission refused (queue or memory full) */
#define AGJ_ECAPACITY     8   /* output or scratch buffer too small for this join */
#define AGJ_EDEVICE       9   /* a device-side bounds check failed (index corrupt) */

const char* agj_strerror(int status);

/* Human-readable reason of the calling thread's last agj_build failure
 * ("" if none); valid until the thread's next agj_build. */
const char* agj_last_error(void);

/* ---------------------------------------------------------------------- */
/* polygons and index build (host)                                          */
/* ---------------------------------------------------------------------- */

/* One polygon: a simple ring of (lat, lng) degree pairs, implicitly closed,
 * either orientation, all on one cube face, optionally with holes.  Edges
 * are geodesics (straight in the face's gnomonic (u,v) plane).  ST_Covers
 * semantics (§II): points on edges and vertices are inside.
 * Holes widen the paper's simple polygons: with n_rings >= 2, latlng holds
 * the outer ring followed by the hole rings, ring q ending (exclusive) at
 * vertex ring_ends[q] (ascending, the last = n_vertices, each ring >= 3
 * vertices).  The polygon is the outer ring minus the interiors of its
 * holes: a point on an edge of any ring is on the boundary, otherwise it is
 * inside when it lies inside an odd number of rings (holes are expected
 * inside the outer ring and disjoint; that rule defines the result anyway).
 * n_rings 0 or 1: a single ring of n_vertices >= 3, ring_ends unused. */
typedef struct {
    uint32_t n_vertices;       /* all rings together */
    uint32_t n_rings;          /* 0 or 1: one ring; k >= 2: the outer ring and k - 1 holes */
    const double* latlng;      /* host, 2 * n_vertices doubles */
    const uint32_t* ring_ends; /* host, n_rings >= 2: n_rings ascending ring ends */
} agj_polygon;

typedef enum {
    AGJ_APPROX = 0,   /* §III-A approximate join: candidate cells refined until
                         their diagonal is below the precision; no PIP */
    AGJ_EXACT  = 1,   /* §III-A exact join: trained index + PIP on candidates */
    AGJ_AUTO   = 2    /* build only: §III-A's choice between the two - the
                         approximate index if it fits memory_budget_bytes
                         (which must be set), else the exact one trained
                         within that budget; agj_index_stats' mode says which */
} agj_mode;

/* Join predicate of the exact join (§II).  The paper joins by ST_Covers and
 * notes that other predicates, naming ST_Intersects, follow with similar
 * techniques.  The index is the same for all three: its true-hit cells lie
 * strictly inside their polygons, so only the refine test of candidate
 * pairs differs, and only for points exactly on a polygon's edge or vertex.
 * The approximate join is the same for every predicate (its extra pairs lie
 * within precision_m, §III-A). */
typedef enum {
    AGJ_COVERS = 0,      /* ST_Covers: points on an edge or vertex are inside (default) */
    AGJ_INTERSECTS = 1,  /* ST_Intersects: a point meets a polygon iff the polygon covers
                            it, so the result equals AGJ_COVERS */
    AGJ_CONTAINS = 2     /* ST_Contains: the interior only; points on an edge or vertex
                            are outside */
} agj_predicate;

/* Build options; zero-initialise and set what you need.  0 selects the
 * default noted beside each field. */
typedef struct {
    uint32_t max_cover_cells;     /* 0 -> 128 (§V defaults) */
    uint32_t max_cover_level;     /* 0 -> 30  */
    uint32_t max_interior_cells;  /* 0 -> 256 */
    uint32_t max_interior_level;  /* 0 -> 20  */
    uint64_t memory_budget_bytes; /* 0 -> unlimited in approx mode; in exact
                                     mode 4x the untrained trie size */
    const double* train_latlng;   /* host, exact mode: training points (§III-D), may be NULL */
    uint64_t n_train;
    uint32_t max_train_level;     /* 0 -> 24 */
    uint32_t n_threads;           /* host build threads, 0 -> all cores */
    uint32_t host_only;           /* 1: build the host index only, no device copy
                                     (for inspection; agj_join then returns AGJ_EINVAL) */
    uint32_t no_fast_ids;         /* 1: always compute cell ids in FP64 (no certified
                                     FP32 model); results are identical, only slower */
    uint32_t no_pip_bands;        /* 1: the certified refine test scans every edge
                                     instead of the point's band; identical results */
    uint32_t predicate;           /* agj_predicate of the exact join, 0 -> AGJ_COVERS;
                                     another value is AGJ_EINVAL */
} agj_build_opts;

typedef struct agj_index agj_index;

/*
 * Builds the logical index (coverings + interior coverings merged by the
 * super-covering listing, §III-B), refines it (approx: candidate cells split
 * until diagonal + 2e-5 m < precision_m, §III-A; exact: training, §III-D),
 * builds the Adaptive Cell Trie and lookup table (§III-C) on the host and
 * copies them, with the polygons' face (u,v) vertices for refinement, to
 * the current device on `stream` (the call synchronises on `stream` before
 * returning).  precision_m is used in approx mode only.
 * Ownership: *out is owned by the caller and released with agj_free.
 * Errors: AGJ_EINVAL (null, a ring with < 3 vertices, ring ends not ascending
 * to n_vertices, invalid vertex, precision_m <= 0 in approx mode, AGJ_AUTO
 * without a memory budget, unknown predicate), AGJ_EUNSUPPORTED
 * (polygon spans faces, too many polygons), AGJ_EBUDGET (approx index above
 * memory_budget_bytes; AGJ_AUTO then builds the exact index instead),
 * AGJ_ENOMEM, AGJ_ECUDA.
 */
int agj_build(const agj_polygon* polys, uint32_t n_polys, double precision_m, agj_mode mode,
              const agj_build_opts* opts, void* stream, agj_index** out);

/* Releases the index and its device memory (synchronises the device). */
void agj_free(agj_index* index);

typedef struct {
    uint32_t mode;             /* agj_mode */
    uint32_t n_polys;
    uint64_t n_cells;          /* logical cells (super covering) */
    uint64_t n_cand_cells;     /* cells with >= 1 candidate reference */
    uint64_t n_nodes;          /* trie nodes (256 x 8 bytes each) */
    uint64_t n_lut_words;      /* lookup-table uint32 words */
    uint64_t device_bytes;     /* bytes resident on the device */
    uint32_t max_refs;         /* largest reference list of a cell */
    uint32_t max_cand_refs;    /* largest candidate list of a cell */
    uint32_t max_depth;        /* deepest trie level below the face roots */
    uint32_t max_level;        /* finest cell level */
    double   build_seconds;
    uint32_t fast_ids;         /* 1: certified FP32 cell-id model in use */
    uint32_t predicate;        /* agj_predicate the index joins by */
    double   fast_err_cells;   /* its error bound, in level-30 cells */
} agj_stats;

int agj_index_stats(const agj_index* index, agj_stats* out);

/*
 * Copies the logical index (the super covering) to host arrays: cells
 * ascending by id, cell k's references refs[ref_off[k] .. ref_off[k+1]) with
 * ref = polygon_id << 1 | interior (§III-B "polygon reference").  Call with
 * NULL arrays to query n_cells and n_refs; then with arrays of those sizes
 * (cells: n_cells, ref_off: n_cells + 1, refs: n_refs).
 */
int agj_index_logical(const agj_index* index, uint64_t* cells, uint64_t* ref_off, uint32_t* refs,
                      uint64_t* n_cells, uint64_t* n_refs);

/*
 * The super-covering merge alone (§III-B, Listing "Build super covering"),
 * for callers that bring their own coverings: inserts (cells[k], refs[k]) in
 * order (ref = polygon_id << 1 | interior); a duplicate cell merges
 * references, an ancestor/descendant conflict replaces the ancestor c1 by
 * the descendant c2 plus the difference cells d (3 per level between them),
 * all carrying c1's references, and c2 also gets the new reference.  When
 * one polygon is referenced both as true and as candidate, true wins.
 * Output: out_cells ascending, out_refs[out_off[k] .. out_off[k+1]).  Call
 * with NULL outputs to get *n_out_cells and *n_out_refs first.  Host only.
 */
int agj_supercover(const uint64_t* cells, const uint32_t* refs, uint64_t n, uint64_t* out_cells, uint64_t* out_off,
                   uint32_t* out_refs, uint64_t* n_out_cells, uint64_t* n_out_refs);

/*
 * The lookup-table encoding (§III-C "Lookup table") the trie uses for
 * cells with more than two references: list k (refs[ref_off[k] ..
 * ref_off[k+1]), ref = polygon_id << 1 | interior, in the caller's order) is
 * stored as [n_true, true ids..., n_cand, candidate ids...] in one uint32
 * array, each distinct list once; offsets[k] = its word offset.  Call with
 * words == NULL to get *n_words first.  Host only.
 */
int agj_lut_encode(const uint32_t* refs, const uint64_t* ref_off, uint64_t n_lists, uint32_t* words,
                   uint64_t* offsets, uint64_t* n_words);

/* Copies the flattened trie to host: nodes (n_nodes * 256 uint64 tagged
 * entries), the lookup table (n_lut_words) and the face table (6 x
 * {root node or 0xFFFFFFFF, prefix length in key bits, prefix}).  NULL arrays
 * are skipped.  The entries' polygon references name the index's pieces:
 * the input polygons themselves unless a polygon crosses cube faces (then
 * it has one piece per face it reaches, numbered in polygon order). */
int agj_index_trie(const agj_index* index, uint64_t* nodes, uint32_t* lut, uint64_t face_table[18]);

/* ---------------------------------------------------------------------- */
/* the probe: join points against an index (device)                         */
/* ---------------------------------------------------------------------- */

/*
 * Output of a join as CSR: the polygon ids joined with point p are
 * ids[offsets[p] .. offsets[p+1]), ascending and unique; offsets[n] = nnz.
 * All buffers are device memory.  `scratch` is device work space used by
 * the join (tile states of the one-pass scan, candidate queues in exact
 * mode); its size comes from agj_join_requirements.
 */
typedef struct {
    uint32_t* offsets;        /* n + 1 */
    uint32_t* ids;            /* ids_capacity */
    uint64_t  ids_capacity;
    void*     scratch;        /* scratch_bytes, 256-byte aligned; after a join its
                                 bytes 16..23 hold the number of points whose
                                 walk recomputed the FP64 cell id and bytes
                                 24..31 the number of candidates whose refine
                                 test fell back to FP64 (diagnostics) */
    uint64_t  scratch_bytes;
    uint64_t* status;         /* 4 x uint64 device words: [0] nnz, [1] error flags,
                                 [2] candidate pairs refined (exact mode),
                                 [3] trie node entries read by the walk */
} agj_pairs;

typedef struct {
    uint64_t ids_capacity;    /* ids that any join of n points can produce */
    uint64_t scratch_bytes;
} agj_requirements;

/* Sizes of the buffers a join of up to n points needs (host only). */
int agj_join_requirements(const agj_index* index, uint64_t n, agj_requirements* out);

/* Allocates an agj_pairs for up to n points with cudaMallocAsync on
 * `stream`; release with agj_pairs_free on a stream ordered after use. */
int agj_pairs_alloc(const agj_index* index, uint64_t n, void* stream, agj_pairs* out);
int agj_pairs_free(agj_pairs* pairs, void* stream);

/*
 * The probe (§III-E, Listing "The probe algorithm"): for each point, its
 * 64-bit cell id, the trie walk from its face root (Listing "Probe Adaptive
 * Cell Trie"), the references of the cell found; approx mode outputs every
 * reference, exact mode outputs true hits and the candidates that pass the
 * FP64 ST_Covers test.  d_points: device, n x {lat, lng}, 16-byte aligned,
 * borrowed.  `out` buffers must satisfy agj_join_requirements(index, n).
 * Asynchronous on `stream`; out->status[0] holds nnz when the stream
 * reaches that point.  n == 0 writes offsets[0] = 0.  n must be < 2^32.
 * Errors (returned immediately): AGJ_EINVAL, AGJ_ECAPACITY (buffers too
 * small for n), AGJ_ECUDA (launch failed).  Device-side conditions are
 * reported in out->status[1] (bit 0 ids capacity exceeded, bit 1 a device
 * wait timed out: the scan's look-back or a probe block's wait for its
 * shared tables, bit 2 trie bounds check, bit 3 candidate queue overflow)
 * and by agj_join_check.
 */
int agj_join(const agj_index* index, const double* d_points, uint64_t n, void* stream, agj_pairs* out);

/*
 * Approximate join that allocates nothing.  The paper has no counterpart;
 * this entry point exists for callers that cannot call cudaMalloc (or any
 * allocating routine) when they join: code running under a device-memory
 * budget that was split up front, plugins hosted by another framework that
 * owns every device allocation, and latency-bound loops where an allocation
 * could synchronise the device and stall other streams.
 *
 * It computes the same CSR as agj_join for an AGJ_APPROX index, with a
 * one-pass kernel built on the same probe and emit helpers (probe, tile
 * scan by look-back, emit); that scan's work space is a static device array
 * of the library, sized for at most AGJ_NOALLOC_MAX_POINTS points per call,
 * held by every device that loads the library until the process exits.
 * The caller passes the inputs and outputs: d_points (device, n x {lat, lng},
 * 16-byte aligned), d_offsets (device, n + 1 uint32), d_ids (device,
 * ids_capacity uint32, at least n * max_refs of agj_index_stats) and
 * d_status (device, 4 uint64 words, same meaning as agj_pairs.status).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.
 * All calls on one device share the array: calls whose kernels overlap on
 * the GPU (different streams, no ordering between them) race and give wrong
 * results; order them on one stream or with events.
 * Errors: AGJ_EINVAL (null or misaligned pointer, exact-mode index, index
 * built with host_only), AGJ_ECAPACITY (n > AGJ_NOALLOC_MAX_POINTS;
 * ids_capacity below n * max_refs; or n * max_refs >= 2^32 - 1, beyond the
 * 32-bit offsets, as for agj_join), AGJ_ECUDA.  Only the first
 * n * max_refs ids are ever written.  Device-side conditions land in
 * d_status[1] as for agj_join.  Asynchronous on `stream`.
 */
#define AGJ_NOALLOC_MAX_POINTS (1ull << 24)
int agj_join_approx_noalloc(const agj_index* index, const double* d_points, uint64_t n, uint32_t* d_offsets,
                            uint32_t* d_ids, uint64_t ids_capacity, uint64_t* d_status, void* stream);

/*
 * agj_join that also records four caller-created CUDA events (cudaEvent_t
 * passed as void*) on `stream` at its stage boundaries, for timing the
 * kernels with cudaEventElapsedTime:
 *   approx: [0] before the probe kernel, [1] after it, [2] after the scan of
 *           the tile counts, [3] after the emit kernel;
 *   exact:  [0] before the probe kernel, [1] after it, [2] after the refine
 *           (grouping + PIP), [3] after the scan and emit kernels.
 * n == 0 records all four events back to back.
 */
int agj_join_timed(const agj_index* index, const double* d_points, uint64_t n, void* stream, agj_pairs* out,
                   void* const events[4]);

/*
 * Aggregation mode: the query the paper benchmarks (§V: the points of a
 * stream joined with a polygon set, "count(*) ... group by polygon_id").
 * The probe is the join's (cell id, face/prefix stage, trie walk, §III-E);
 * instead of pairs it adds every counted reference to its polygon, as the
 * SIMD aggregation of §IV does with gather/scatter: the lanes of a warp
 * that name the same polygon are combined into one add, and the rare
 * lanes (cells with more than two references; in exact mode candidate
 * references) are handled apart.  In exact mode the candidates are refined
 * by the same ST_Covers step as agj_join, grouped by polygon, and each
 * group's passes are added at once.
 *
 * Result: d_counts[P] (device, n_polys uint64) = the number of points p of
 * this call for which agj_join on the same index and points would output
 * the pair (p, P), i.e. the number of times P occurs in its ids; with
 * accumulate != 0 these are added to d_counts, else d_counts is
 * overwritten.  d_status (device, 4 uint64 words): [0] pairs counted (the
 * sum of this call's counts), [1] error flags as for agj_join (bit 1 scan
 * wait timed out, bit 2 trie bounds check, bit 3 candidate queue
 * overflow), [2] candidate pairs refined (exact mode), [3] trie node
 * entries read.  d_points: device, n x {lat, lng}, 16-byte aligned,
 * borrowed; n < 2^32.  d_scratch: device work space of at least
 * agj_count_scratch_bytes(index, n) bytes, 256-byte aligned (bytes 16..23
 * receive the count of points whose walk recomputed the FP64 cell id,
 * 24..31 the count of candidates refined in FP64).  Asynchronous on
 * `stream`.  Errors (returned immediately): AGJ_EINVAL (null or misaligned
 * pointer, n >= 2^32, index built with host_only), AGJ_ECAPACITY (scratch
 * too small, or the exact candidate queue beyond 32-bit slots), AGJ_ECUDA.
 */
uint64_t agj_count_scratch_bytes(const agj_index* index, uint64_t n);
int agj_join_count(const agj_index* index, const double* d_points, uint64_t n, void* stream, uint64_t* d_counts,
                   int accumulate, uint64_t* d_status, void* d_scratch, uint64_t scratch_bytes);
/* agj_join_count recording four caller-created events on `stream`: [0]
 * before the probe kernel, [1] after it, [2] after the refine (exact mode;
 * right after [1] in approx mode), [3] at the end. */
int agj_join_count_timed(const agj_index* index, const double* d_points, uint64_t n, void* stream, uint64_t* d_counts,
                         int accumulate, uint64_t* d_status, void* d_scratch, uint64_t scratch_bytes,
                         void* const events[4]);

/*
 * Training from a point stream on the device (§III-D; the paper trains
 * offline and leaves online training to future work).  The probe kernels
 * walk n device points (n x {lat, lng}, 16-byte aligned) and return to the
 * host only those that land in a cell with candidate references (the
 * "expensive" cells training refines); the host splits those cells in
 * descending order of hits within memory_budget_bytes of trie nodes (0: four
 * times the current trie), as agj_build's training does, re-flattens the
 * trie and replaces the index's device copy.  Points outside the expensive
 * cells cannot change training, so the result is the index agj_build
 * would produce from the same polygons and these training points.  Exact
 * mode only.  The join results do not change (exact mode), only how many
 * candidates need the refine step.  Synchronises the device; no join on
 * this index may be in flight.  Errors: AGJ_EINVAL (not an exact index on
 * the device, misaligned or null points, n >= 2^32), AGJ_EDEVICE, AGJ_ENOMEM
 * (the index then keeps no device copy), AGJ_ECUDA.
 */
int agj_train_online(agj_index* index, const double* d_points, uint64_t n, uint64_t memory_budget_bytes,
                     void* stream);

/* ---------------------------------------------------------------------- */
/* batched form (no counterpart in the paper)                               */
/* ---------------------------------------------------------------------- */

/*
 * A plan that joins m (index, point batch) jobs of uneven sizes in one
 * launch sequence: the probe and emit kernels cover every job's warp tiles
 * (one warp per tile, or persistent grids striding over them), the refine
 * step covers the candidates of all exact jobs at once, and the sequence is
 * captured once into a CUDA graph that each run replays.  In a large plan
 * with both modes the approximate and the exact jobs run as two independent
 * chains of kernels compiled for their mode, parallel branches of the graph.
 * The paper joins one point stream against one
 * index; the batched form serves callers with many small or uneven batches,
 * where one plain join per batch pays a launch sequence and a grid tail per
 * batch.
 *
 * Every job computes exactly what agj_join computes for the same (index,
 * points) - the same pairs, ids ascending per point, the same status words.
 *
 * agj_batch_create: indexes[j] (built on the current device, not host_only)
 * and n[j] (< 2^32 points) fix the plan; the points and outputs are given
 * per run.  opts may be NULL (defaults).  The plan owns one device
 * allocation (work space for all jobs, agj_batch_device_bytes) and, with
 * use_graph, an instantiated graph.  At most 65535 jobs (AGJ_EUNSUPPORTED
 * beyond).  Errors: AGJ_EINVAL (null or foreign index, bad option),
 * AGJ_ECAPACITY (a job's ids or the candidate queue
 * would not fit 32-bit offsets), AGJ_ENOMEM, AGJ_ECUDA.
 */
typedef struct agj_batch agj_batch;
typedef struct {
    uint32_t points_per_lane;   /* 1, 2 or 4 points per lane of a warp tile (0 = 2) */
    uint32_t ctas_per_sm;       /* 0: one warp per warp tile of all jobs; 1..8: persistent
                                   probe grid of SMs x this CTAs */
    uint32_t no_graph;          /* 1: enqueue the kernels on each run instead of a graph */
    uint32_t reserved;
} agj_batch_opts;
int agj_batch_create(const agj_index* const* indexes, const uint64_t* n, uint32_t m, const agj_batch_opts* opts,
                     agj_batch** out);

/*
 * Runs the plan: d_points[j] (device, n[j] x {lat, lng}, 16-byte aligned,
 * borrowed) joined into outs[j], whose offsets, ids and status must satisfy
 * agj_join_requirements(indexes[j], n[j]) (scratch is not needed: when
 * outs[j].scratch is given with at least 32 bytes, its bytes 16..31 receive
 * the job's diagnostics as agj_join writes them).  Asynchronous on
 * `stream`; runs of one plan must be ordered (one stream), as they share its
 * work space.  Errors: AGJ_EINVAL, AGJ_ECAPACITY, AGJ_ECUDA; device-side
 * conditions land in outs[j].status[1] as for agj_join.
 */
int agj_batch_run(agj_batch* batch, const double* const* d_points, void* stream, agj_pairs* outs);
uint64_t agj_batch_device_bytes(const agj_batch* batch);
/* Frees the plan; the caller orders it after the plan's last run. */
void agj_batch_free(agj_batch* batch);

/*
 * One-shot batched join: creates a plan with default options, runs it on
 * `stream`, synchronises the stream and frees the plan.
 */
int agj_join_batched(const agj_index* const* indexes, const double* const* d_points, const uint64_t* n,
                     uint32_t m, void* stream, agj_pairs* outs);

/* ---------------------------------------------------------------------- */
/* served form (no counterpart in the paper)                                */
/* ---------------------------------------------------------------------- */

/*
 * A request loop over resident indexes.  The paper motivates low-latency
 * joins for streaming points but measures none; this form serves many small
 * point requests by continuous batching: a scheduler thread forms a launch
 * from the requests waiting whenever one of its n_slots slots (streams) is
 * free and runs it as one batched join (see agj_batch_create) on that
 * slot's stream while other slots' launches are in flight.  Each request's
 * result is exactly what agj_join computes for its points.  Request points
 * are read by the probe kernels from the client's host buffer where the
 * device can read pageable host memory (see AGJ_SERVER_STAGE_POINTS), else
 * staged; results come back through the slot's pinned buffers.
 *
 * Admission by device memory: the launches in flight share one device
 * arena of hbm_budget_bytes.  A launch takes the exact bytes of its points,
 * outputs and join work space from the arena (first fit); the scheduler
 * takes requests from the queue head up to max_step_points /
 * max_step_requests and cuts the launch back until it fits a free block,
 * and when not even the head request fits it waits for a launch in flight
 * to finish and return its block (counted in memory_waits).  Indexes are
 * admitted against the free device memory by agj_server_add_index.
 *
 * agj_server_create: indexes (built on the current device) are borrowed and
 * must outlive the server; requests name them by position.  opts may be
 * NULL.  The arena is hbm_budget_bytes, or (0) room for n_slots launches of
 * max_step_points points, in either case no more than the device's free
 * memory less hbm_reserve_bytes (AGJ_EBUDGET if a given budget exceeds
 * that).  Errors: AGJ_EINVAL, AGJ_EBUDGET, AGJ_ENOMEM, AGJ_ECUDA.
 */
typedef struct agj_server agj_server;
typedef struct {
    uint32_t n_slots;            /* launches in flight, 0 = 4 */
    uint32_t max_step_requests;  /* requests per launch (<= 65535), 0 = 4096 */
    uint64_t max_step_points;    /* points per launch (and per request), 0 = 2^20 */
    uint64_t hbm_budget_bytes;   /* device arena for the launches in flight, 0 = see above */
    uint64_t max_pending;        /* queued requests before submit answers AGJ_EBUSY, 0 = 2^20 */
    uint32_t points_per_lane;    /* as agj_batch_opts, 0 = 2 */
    uint32_t ctas_per_sm;        /* as agj_batch_opts */
    uint32_t flags;              /* AGJ_SERVER_STAGE_POINTS */
    uint32_t max_refs;           /* largest reference list of an index added later by
                                    agj_server_add_index (sizes the pinned id buffers);
                                    0 = that of the indexes given at creation */
    uint64_t hbm_reserve_bytes;  /* free device memory admission leaves untouched, 0 = 1 GiB */
} agj_server_opts;
/* Where the device can read pageable host memory (GB300: NVLink-C2C with
 * the host's page tables), the probe reads each request's points straight
 * from the client's buffer; this flag copies them through pinned staging
 * buffers and one host-to-device copy per launch instead. */
#define AGJ_SERVER_STAGE_POINTS 1u
int agj_server_create(const agj_index* const* indexes, uint32_t n_indexes, const agj_server_opts* opts,
                      agj_server** out);

/*
 * Queues a request: h_points (host, n x {lat, lng}) is borrowed until the
 * request completes.  With h_offsets (host, n + 1) and h_ids (host,
 * ids_capacity) the result is written there and kept until
 * agj_server_poll; with both NULL the result is discarded and only counted
 * in the statistics.  *ticket names the request.  Errors: AGJ_EINVAL,
 * AGJ_ECAPACITY (n > max_step_points), AGJ_EBUDGET (the request alone
 * would not fit the arena), AGJ_EBUSY (max_pending queued).
 */
int agj_server_submit(agj_server* server, uint32_t index_id, const double* h_points, uint64_t n,
                      uint32_t* h_offsets, uint32_t* h_ids, uint64_t ids_capacity, uint64_t* ticket);

/*
 * Admits one more index (no counterpart in the paper): an index built with
 * host_only = 1 is uploaded to the device (becoming as if built there; it
 * stays resident until agj_free) if its device blob fits the device's free
 * memory less hbm_reserve_bytes, else AGJ_EBUDGET and nothing changes; an
 * index already on the server's device is added as it is.  *index_id
 * receives its position for agj_server_submit.  Safe while requests are in
 * flight.  The index must outlive the server.  Errors: AGJ_EINVAL,
 * AGJ_EBUDGET, AGJ_ECAPACITY (its largest reference list exceeds the
 * server's max_refs), AGJ_EUNSUPPORTED (4096 indexes), AGJ_ENOMEM,
 * AGJ_ECUDA.
 */
int agj_server_add_index(agj_server* server, agj_index* index, uint32_t* index_id);

typedef struct {
    int32_t  status;             /* AGJ_OK, or the request's error */
    uint32_t reserved;
    uint64_t nnz;                /* pairs of the request */
    uint64_t t_submit_ns, t_start_ns, t_done_ns;   /* steady clock */
    uint64_t step;               /* launch that served it (1, 2, ...) */
} agj_request_result;

/* Result of a kept request (wait != 0 blocks until it completes; else
 * AGJ_EBUSY while it runs).  A polled result is released. */
int agj_server_poll(agj_server* server, uint64_t ticket, int wait, agj_request_result* out);
/* Blocks until every submitted request has completed. */
int agj_server_drain(agj_server* server);

typedef struct {
    uint64_t submitted, completed, rejected, points, steps, step_requests_max;
    uint32_t n_slots;
    uint32_t host_reads;         /* 1: the probe reads request points from host memory */
    uint64_t device_bytes;       /* the launches' device arena */
    double p50_us, p99_us, mean_us, max_us;   /* submit-to-done latency of completed requests */
    uint64_t memory_waits;       /* times the scheduler waited for arena memory */
    uint64_t peak_bytes_in_use;  /* largest arena use by the launches in flight */
    uint64_t index_bytes;        /* device bytes of the indexes agj_server_add_index uploaded */
    uint32_t n_indexes;
    uint32_t reserved;
} agj_server_stats;
/* Statistics since creation or the last reset (reset != 0 clears them). */
int agj_server_get_stats(agj_server* server, int reset, agj_server_stats* out);
/* Drains, stops the scheduler and frees the server. */
void agj_server_destroy(agj_server* server);

/*
 * Poisson load for the served form: n_requests arrivals at `rate` per
 * second; sizes 1..max_points with P(k) proportional to k^-zipf_alpha; each
 * addresses a uniformly drawn set, its exact index with probability
 * exact_fraction (when exact_index[set] != 0xFFFFFFFF), else its approximate
 * index; its points are a random contiguous slice of the set's host pool
 * (pool_points[set] >= max_points).  The first warmup_requests are left
 * out of the statistics.
 */
typedef struct {
    double rate;
    uint64_t n_requests;
    double zipf_alpha;
    uint32_t max_points;
    uint32_t n_sets;
    double exact_fraction;
    const uint32_t* approx_index;
    const uint32_t* exact_index;
    const double* const* pools;
    const uint64_t* pool_points;
    uint64_t seed;
    uint64_t warmup_requests;
} agj_load_spec;
typedef struct {
    uint64_t requests, points, rejected;
    double seconds, offered_rate, achieved_rate, points_per_s;
    double p50_us, p99_us, mean_us, max_us;   /* arrival-to-done latency */
} agj_load_result;
/* Drives `server` with the spec's arrivals (submitting at arrival times
 * from the calling thread) and waits for all of them. */
int agj_server_load(agj_server* server, const agj_load_spec* spec, agj_load_result* out);
/* The same arrivals served one at a time by agj_join_host (the plain join
 * of a host request) in arrival order, for comparison; index ids name
 * positions in `indexes`. */
int agj_plain_load(const agj_index* const* indexes, uint32_t n_indexes, const agj_load_spec* spec,
                   agj_load_result* out);

/* Synchronises `stream`, reads out->status and returns AGJ_OK, or the first
 * device-side error as a status code; *nnz receives the pair count. */
int agj_join_check(const agj_pairs* pairs, void* stream, uint64_t* nnz);

/*
 * End-to-end join from host memory: h_points (n x {lat, lng}) are read by
 * the probe where they are when the device can read them (pinned memory, or
 * pageable memory on devices that read the host's page tables, as GB300 over
 * NVLink-C2C; 16-byte aligned) and copied to d_points_staging (device, n x 16
 * bytes; may be NULL when not needed) otherwise; the CSR comes back to
 * h_offsets (n + 1) and h_ids (up to h_ids_capacity).  Uses `work` (from
 * agj_pairs_alloc or caller buffers for n points).  Synchronises `stream`.
 * *nnz receives the pair count; AGJ_ECAPACITY if h_ids is too small
 * (h_offsets is still filled).
 */
int agj_join_host(const agj_index* index, const double* h_points, uint64_t n, double* d_points_staging,
                  agj_pairs* work, uint32_t* h_offsets, uint32_t* h_ids, uint64_t h_ids_capacity,
                  uint64_t* nnz, void* stream);

/*
 * Self-test of the join's bounded device-side waits (no counterpart in the
 * paper).  The tile scan chains CTA chunks by a look-back that waits for
 * each predecessor's published state, with a bounded spin after which it
 * sets the "scan wait timed out" bit of the join's status instead of
 * hanging.  This runs the scan as the second chunk while the first never
 * publishes: it returns AGJ_ETIMEOUT when the wait ran out and was
 * reported (the expected outcome, after about a second), AGJ_OK if it was
 * not, AGJ_ENOMEM / AGJ_ECUDA on setup errors.  The context stays usable.
 * Synchronises `stream`.
 */
int agj_selftest_scan_timeout(void* stream);

/*
 * Self-test of the probe's bounded wait for its block's shared tables (no
 * counterpart in the paper).  A probe block stages the Hilbert table and
 * the trie's root node in shared memory with asynchronous copies that
 * arrive on a block-local barrier; each warp waits on that barrier with a
 * bounded loop (about a second), after which its tile joins nothing and the
 * join's status[1] gets bit 1 (a device wait timed out).  This stages the
 * tables on a barrier expecting one arrival too many: it returns
 * AGJ_ETIMEOUT when the wait ran out and was reported (the expected
 * outcome), AGJ_OK if it was not, AGJ_ENOMEM / AGJ_ECUDA on setup errors.
 * The context stays usable.  Synchronises `stream`.
 */
int agj_selftest_ready_timeout(void* stream);

/*
 * Measurement utility (no counterpart in the paper): the FP64 fused
 * multiply-add rate of the current device in flop/s (2 per FMA), from the
 * library's own kernel of independent FMA chains on every SM, best of five
 * timed launches.  The cell-id kernel's FP64 roofline is stated against
 * it.  Allocates 64 bytes of device memory and synchronises `stream`.
 */
int agj_measure_fp64_rate(void* stream, double* flops_per_s);

/* Cell ids of points with the device kernel (FP64 spec, bit-exact); for
 * checking the id step alone.  d_ids: device, n uint64. */
int agj_cell_ids(const double* d_points, uint64_t n, uint64_t* d_ids, void* stream);

/*
 * The certified fast cell-id step on the host, with the same FP32 model and
 * arithmetic the probe kernels use (agj_stats.fast_ids must be 1): for each
 * point, h_levels[k] = 255 if the point lies outside the model's window (it
 * joins nothing), else the number L of leading levels (0..30) whose digits
 * are certified equal to the FP64 spec's, and h_ids[k] = the leaf id built
 * from the model's (i, j): its first L levels equal the spec id's.
 * AGJ_EUNSUPPORTED if the index has no fast model.  Host only.
 */
int agj_fast_ids_host(const agj_index* index, const double* h_points, uint64_t n, uint64_t* h_ids,
                      uint8_t* h_levels);

/*
 * The certified FP32 refine test on the host, with the same model and
 * arithmetic the PIP kernel uses: for point k and polygon h_polys[k],
 * h_out[k] = 1 (covered), 0 (not covered) or -1 (undecided: the kernel then
 * recomputes the test in FP64).  A polygon across cube faces is tested as
 * its piece on the point's face (0 when it has none there).  Host only.
 */
int agj_covers_certified_host(const agj_index* index, const double* h_points, const uint32_t* h_polys, uint64_t n,
                              int8_t* h_out);

/* Cell ids of points on the host with the same spec (host code). */
int agj_cell_ids_host(const double* h_points, uint64_t n, uint64_t* h_ids);

#ifdef __cplusplus
}
#endif

#endif /* AGJ_H */
