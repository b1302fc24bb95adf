/*
 * msc.h -- C ABI of libmsc, a GPU (sm_103a) implementation of the iterative edit loop of
 * "Preserving Discrete Morse-Smale Complexes in Error-Bounded Lossy Compression"
 * (Li, Xia, Liang, Wang, Guo): given an original scalar field f and a base compressor's
 * decompressed field f_hat on the same regular grid, compute per-vertex edits so that the
 * edited field g = f_hat + delta satisfies |f - g| <= xi and has the same discrete
 * Morse-Smale complex as f (Sec. 4.1, "Problem Statement").
 *
 * Conventions used by every entry point
 *  - Grid: nx x ny x nz vertices, nz == 1 for a 2D field; vertex id v = x + nx*(y + ny*z)
 *    (x fastest).  nx, ny >= 2, nz >= 1, and nx*ny*nz < 2^31.
 *  - Complex: the Freudenthal triangulation of the grid (Sec. 4.8.1: six tetrahedra per
 *    cube in 3D, two triangles per square in 2D), with the diagonal along +(1,1[,1]).
 *  - Vertex order: simulation of simplicity (Sec. 4.1, "Degeneracy handling"): a < b iff
 *    f[a] < f[b], or f[a] == f[b] and a < b.
 *  - Field pointers may be host or device memory; the library finds out with
 *    cudaPointerGetAttributes.  Device pointers must be on the current device.
 *  - Ownership: the caller owns every input and every output buffer it passes (g_out,
 *    rows).  The library owns a handle and the arrays inside msc_edits; free them with
 *    msc_destroy / msc_free_edits.
 *  - Errors: every call returns a status and never aborts.  On any status other than
 *    MSC_OK the outputs are unspecified; msc_last_error() gives a one-line reason
 *    (thread-local, valid until the next call on the same thread).
 *  - Streams: options->stream (a cudaStream_t, NULL = the legacy default stream) orders
 *    all device work of a call; calls return after their results are complete.
 */
#ifndef MSC_H
#define MSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msc_handle msc_handle;   /* opaque: device-resident MSC state of one f */

typedef enum {
    MSC_OK = 0,
    MSC_ERR_INVALID_ARG = 1,     /* bad dims, NaN/Inf values, xi <= 0, q_max or tier out of range */
    MSC_ERR_OOM = 2,             /* device or host allocation failed */
    MSC_ERR_CUDA = 3,            /* a CUDA runtime call failed (message in msc_last_error) */
    MSC_ERR_NOT_CONVERGED = 4,   /* max_iters edit rounds were not enough */
    MSC_ERR_DEVICE_TIMEOUT = 5,  /* a bounded device-side wait gave up */
    MSC_ERR_STALLED = 6,         /* every false case targets a vertex that cannot move and
                                    exact_fallback is off */
    MSC_ERR_NO_DEVICE = 7,       /* no CUDA device, or the library was not built for it */
    MSC_ERR_CANCELLED = 8,       /* a serving job cancelled by msc_server_cancel */
    MSC_ERR_UNAVAILABLE = 9      /* a runtime dependency is missing (the zstd library) */
} msc_status;

/* per-vertex edit states (the value of msc_edits.q_map[v] is derived from these) */
#define MSC_QMAP_LOSSLESS 0xFF

typedef struct {
    int tier;            /* 1..4 (Sec. 4.1): 1 extrema, 2 all critical cells,
                            3 + saddle-extremum connectivity, 4 + separatrix geometry */
    int q_max;           /* 1..7: edit step xi / 2^q_max, at most q_max quantised steps (Eq. 2) */
    int max_iters;       /* edit rounds before MSC_ERR_NOT_CONVERGED (default 100000) */
    int exact_fallback;  /* 1 (default): a false case whose target vertex cannot move any
                            more (already at its floor f - xi, or restored) restores the
                            closed 1-rings of the case cell's vertices to f exactly */
    int tile_x, tile_y, tile_z;   /* tile of the dense gradient of 3D fields: 32 x {4,8,16} x {8,16,32}
                                     anchors as instantiated (msc_tile_report lists them);
                                     0, 0, 0 (default) = the autotuned shape */
    void *stream;        /* cudaStream_t for all device work of the call (NULL = default) */
    int record_trace;    /* 1: fill msc_edits.trace with one record per edit round */
    int profile;         /* bitmask of kernel classes (bit k = class k below; MSC_PROFILE_ALL =
                            every class): the launches of those classes are timed with CUDA
                            events on the call's stream and summed into the handle's msc_stats.
                            0 (default) times nothing. */
    int small_round;     /* edit rounds that follow a round which edited fewer than this many
                            vertices run in the persistent round kernel, the others as captured
                            graph nodes: 0 (default) = 8192; 1 = every round as graph nodes.
                            Results do not depend on it. */
    int edit_mode;       /* MSC_EDITS_QUANTIZED (0, default): Eq. 2, at most q_max steps of
                            xi / 2^q_max, then the floor; MSC_EDITS_FLOAT (1): the floating
                            edits the paper compares against (Sec. 4.7): the same steps with no
                            cap on their number (a vertex snaps to the floor only when the next
                            step would pass f - xi), and every edited vertex stored losslessly
                            as an (index, value) pair; q_max must then be 1..6 */
    int cluster_round;   /* of the rounds that run in the persistent round kernel, those that
                            follow a round which edited fewer than this many vertices run in one
                            thread-block cluster (hardware barriers between their phases):
                            0 (default) = 1024; 1 = never.  Results do not depend on it. */
} msc_options;

#define MSC_EDITS_QUANTIZED 0
#define MSC_EDITS_FLOAT 1

/* kernel classes of msc_stats */
enum {
    MSC_K_DENSE = 0,     /* dense discrete gradient of a whole field (Sec. 4.2) */
    MSC_K_CPASS = 1,     /* false critical cells -> targets (Sec. 4.3) */
    MSC_K_EDIT = 2,      /* quantised edit (Eq. 2) + dirty-anchor marking */
    MSC_K_REFRESH = 3,   /* gradient of the anchors around edited vertices */
    MSC_K_REBUILD = 4,   /* mismatch-list rebuild and set clears */
    MSC_K_SEP_INIT = 5,  /* separatrix state: first build of an S-pass (Sec. 4.4) */
    MSC_K_SEP_UPDATE = 6,/* separatrix state: updates around edits; full walks (tier 3) */
    MSC_K_SEP_TARGETS = 7,/* troublemakers from the separatrix state */
    MSC_K_OTHER = 8,     /* initialisation, seeds, output encoding, checks */
    MSC_K_SEP_SEED = 9,  /* separatrix state: propagation from the seeds in the first build */
    MSC_K_ROUNDS = 10,   /* persistent kernel running the C-pass rounds that edit few vertices
                            (targets, edits, refresh and rebuild of each round in one launch) */
    MSC_K_COUNT = 11
};
#define MSC_PROFILE_ALL ((1 << MSC_K_COUNT) - 1)

/* per-handle launch statistics (msc_get_stats); times only for the classes in options.profile */
typedef struct {
    uint64_t launches[12];       /* kernel launches by class, always counted */
    double ms[12];               /* summed CUDA-event duration by class (profiled calls) */
    uint64_t timed_launches[12]; /* launches that were timed */
    uint64_t items[12];          /* work items processed by class: anchors (dense, separatrix
                                    init), anchors with differing critical cells (cpass),
                                    targeted vertices (edit), refreshed anchors (refresh),
                                    dirty anchors (rebuild), node steps (separatrix seed and
                                    update), rounds run (rounds); work done inside the
                                    persistent round kernel is counted in round_work instead */
    uint64_t round_work[3];      /* inside the persistent round kernel: targeted vertices,
                                    refreshed (and rebuilt) anchors, anchors with differing
                                    critical cells visited by the C-pass */
    double round_phase_ms[4];    /* persistent round kernel, device clock of its first block:
                                    C-pass with the targets' edits, decision and restores, order
                                    changes, refresh and rebuild (each up to the end of its
                                    barrier) */
    uint64_t cluster_launches;   /* launches of the round kernel's cluster form (counted also
                                    in launches[MSC_K_ROUNDS]) and the rounds they ran */
    uint64_t cluster_rounds;
} msc_stats;

/* one edit round: kind 0 = C-pass (false critical cells), 1 = S-pass (separatrices);
 * T = vertices lowered by a quantised step this round, X = vertices restored to f */
typedef struct {
    int32_t kind;
    int32_t t_us;                     /* device clock when the round's targets were counted,
                                         microseconds after the first round's */
    int64_t n_targets, n_exact;
    int64_t sum_targets, sum_exact;   /* sums of vertex ids, an order-free digest */
} msc_iter_record;

typedef struct {
    uint64_t n_vertices;
    uint32_t n_iters_c;          /* C-pass edit rounds (Sec. 4.3) */
    uint32_t n_iters_s;          /* S-pass edit rounds (Sec. 4.4) */
    uint32_t n_fallback_iters;   /* rounds in which the exact fallback restored vertices */
    uint32_t reserved;
    uint64_t n_quant;            /* vertices with 1..q_max quantised edits */
    uint64_t n_lossless;         /* vertices stored losslessly (floor, restored, re-clamped) */
    uint8_t *q_map;              /* n_vertices entries: q in 0..q_max (g = f_hat - q*xi/2^q_max,
                                    computed as one float subtraction of fl(q * step)), or
                                    MSC_QMAP_LOSSLESS (g stored in lossless_val) */
    uint64_t *lossless_idx;      /* n_lossless vertex ids, ascending */
    float *lossless_val;         /* final g at those vertices */
    uint32_t n_trace;            /* number of records in trace (record_trace = 1) */
    msc_iter_record *trace;
    double loop_ms;              /* device time of the fix loop (init to convergence) */
} msc_edits;

typedef struct {
    uint64_t fp[4];              /* false positive critical cells by dimension */
    uint64_t fn[4];              /* false negative critical cells by dimension */
    uint64_t sep_mismatch[3];    /* separatrices with a pair missing from g's gradient:
                                    descending, ascending, saddle-saddle (per 2-saddle) */
    uint64_t term_mismatch[2];   /* descending / ascending separatrices ending elsewhere */
    double max_abs_err;          /* max |g - f| */
    int pass;                    /* pass_tier[3]: the full MSC (tier 4) is preserved */
    int pass_tier[4];            /* pass_tier[t-1] = 1 iff max_abs_err <= xi and tier t holds:
                                    1 no false extremum, 2 no false critical cell,
                                    3 + no separatrix ending elsewhere,
                                    4 + no separatrix pair missing from g's gradient */
    int reserved;
} msc_report;

/* Library version string. */
const char *msc_version(void);

/* Human-readable name of a status. */
const char *msc_status_string(msc_status s);

/* One-line description of the last error on this thread ("" if none). */
const char *msc_last_error(void);

/* Fill *opt with defaults: tier 4, q_max 6, max_iters 100000, exact_fallback 1,
 * tiles 0, stream NULL, record_trace 0, profile 0, small_round 0, edit_mode quantized,
 * cluster_round 0. */
void msc_default_options(msc_options *opt);

/* Sec. 4.2 (discrete gradient of f), Sec. 3.1 (critical cells, gradient paths): compute
 * and keep on the device the gradient of the original field f, its critical cells and the
 * seeds of its separatrices.  f: nx*ny*nz floats (host or device), all finite.
 * On MSC_OK *out is a new handle (free with msc_destroy). */
msc_status msc_prepare_original(const float *f, int nx, int ny, int nz,
                                const msc_options *opt, msc_handle **out);

/* Sec. 4.2-4.7: the fix loop.  f_hat: the decompressed field (same grid, host or device,
 * finite; values outside [f - xi, f + xi] are first re-clamped into the bound).  xi > 0
 * is the absolute error bound.  Alternates C-passes (Sec. 4.3) and, for tier >= 3,
 * S-passes (Sec. 4.4) until no false case remains; each pass lowers the target vertices
 * by one quantised step (Eq. 2).  Writes the edited field to g_out (nx*ny*nz floats, host
 * or device, caller-owned) and the edits to *out (library-owned arrays; msc_free_edits).
 * opt may be NULL (defaults). */
msc_status msc_fix(msc_handle *h, const float *f_hat, float xi, const msc_options *opt,
                   msc_edits *out, float *g_out);

/* Sec. 4.7 / Fig. 5 (decompression side): rebuild g from f_hat and stored edits,
 * bit-exactly equal to msc_fix's g_out.  f_hat and g_out: host or device. */
msc_status msc_apply_edits(const float *f_hat, int nx, int ny, int nz, float xi, int q_max,
                           const msc_edits *edits, float *g_out);

/* Sec. 4.7: the edit record as a compact byte stream (the "fixed number of bits per
 * quantised count" that the paper then hands to a dictionary coder; no such coder here).
 * Layout, little-endian: a 32-byte header ("MSCE", version 1, q_max, b, 0, n_vertices u64,
 * n_lossless u64, 0 u64); the q-map at b bits per vertex, b the least number of bits that
 * holds q_max + 2 values, in groups of 8 vertices stored as b bytes (vertex 8k+j in bits
 * [j*b, j*b+b) of group k's little-endian integer), a lossless vertex written as 2^b - 1;
 * then the n_lossless float32 values in increasing vertex order (the vertices themselves are
 * implied by the escape codes).  Size: 32 + ceil(n/8)*b + 4*n_lossless bytes. */
uint64_t msc_packed_bytes(uint64_t n_vertices, uint64_t n_lossless, int q_max);

/* Pack edits (as returned by msc_fix with the same q_max) into out (host or device, cap
 * bytes); *n_out receives the record's size.  out == NULL with cap == 0 only reports the
 * size.  Errors: MSC_ERR_INVALID_ARG for a short buffer, a count above q_max, or
 * lossless_idx not listing exactly the q-map's lossless vertices in increasing order. */
msc_status msc_pack_edits(const msc_edits *e, int q_max, uint8_t *out, uint64_t cap, uint64_t *n_out);

/* Unpack a record of size bytes (host or device) into *out (host arrays, free with
 * msc_free_edits after any return) and its q_max.  n_quant is recomputed; the iteration
 * counts and the trace are not part of the record and read 0.  Errors: MSC_ERR_INVALID_ARG
 * for a malformed record. */
msc_status msc_unpack_edits(const uint8_t *buf, uint64_t size, msc_edits *out, int *q_max);

/* Floating edits as key-value pairs (Sec. 4.7: the form that stores every edit as a float,
 * with its vertex index).  Layout, little-endian: a 32-byte header ("MSCE", version 2, 0, 0,
 * 0, n_vertices u64, n_pairs u64, 0 u64), the n_pairs vertex ids as u32 in increasing order,
 * then the n_pairs float32 values.  Size: 32 + 8 * n_pairs bytes. */
uint64_t msc_kv_bytes(uint64_t n_pairs);

/* Pack the edits of a fix run with edit_mode MSC_EDITS_FLOAT (n_quant must be 0) as
 * key-value pairs into out (host memory, cap bytes); *n_out receives the size (out NULL and
 * cap 0 only report it).  Errors: MSC_ERR_INVALID_ARG for quantised counts, a short buffer or
 * lossless_idx not increasing. */
msc_status msc_pack_edits_kv(const msc_edits *e, uint8_t *out, uint64_t cap, uint64_t *n_out);

/* Unpack a key-value record (host memory) into *out (q_map 0 or MSC_QMAP_LOSSLESS, the pairs;
 * free with msc_free_edits after any return).  msc_apply_edits then rebuilds g from it. */
msc_status msc_unpack_edits_kv(const uint8_t *buf, uint64_t size, msc_edits *out);

/* Sec. 4.7 / Sec. 5.5: the lossless coder the paper applies to edit records (ZSTD).  The
 * system's zstd library is loaded on first use; every call returns MSC_ERR_UNAVAILABLE (and
 * msc_coded_bound 0) where it cannot be loaded.  All buffers are host memory.
 *  msc_coded_bound: the largest coded size of a size-byte record (the size out must have).
 *  msc_code_record: code rec[0, size) as one zstd frame at level 1..22 (3 is zstd's default)
 *    into out; *n_out receives the coded size.
 *  msc_decoded_size: the record size stored in a coded frame's header.
 *  msc_decode_record: decode a frame into out (at least msc_decoded_size bytes).
 * Errors: MSC_ERR_INVALID_ARG for a bad level, a short buffer or a damaged frame. */
uint64_t msc_coded_bound(uint64_t size);
msc_status msc_code_record(const uint8_t *rec, uint64_t size, int level, uint8_t *out, uint64_t cap, uint64_t *n_out);
msc_status msc_decoded_size(const uint8_t *in, uint64_t size, uint64_t *n_out);
msc_status msc_decode_record(const uint8_t *in, uint64_t size, uint8_t *out, uint64_t cap, uint64_t *n_out);

/* Sec. 5.1 metrics: compare the MSC of g with the handle's original (critical cells by
 * dimension, every separatrix pair, separatrix terminals) and measure max |g - f|.
 * g: host or device.  Separatrix counts are computed only when the critical cells agree. */
msc_status msc_verify(msc_handle *h, const float *g, float xi, msc_report *out);

/* Free the arrays inside *e (not e itself) and zero it. */
void msc_free_edits(msc_edits *e);

/* Free a handle and its device memory. */
void msc_destroy(msc_handle *h);

/* Batched fix (Sec. 5, time-series study): n independent jobs, job i on handle hs[i] with
 * decompressed field f_hats[i], bound xis[i], outputs outs[i] and g_outs[i] (same rules
 * as msc_fix).  Up to 8 jobs run at once, each on its own stream driven by its own host
 * thread, so their rounds overlap on the device; the jobs start after the work already
 * queued on opt->stream and are all finished when the call returns.  Each job's results
 * equal those of a separate msc_fix call.  The handles must be distinct.  Returns
 * MSC_OK, or the status of the lowest-numbered failing job (the other jobs still run). */
msc_status msc_fix_batch(msc_handle **hs, const float **f_hats, const float *xis, int n,
                         const msc_options *opt, msc_edits *outs, float **g_outs);

/* Sec. 4.2: every gradient pair (L, U) of a field, as rows of 8 int64 vertex ids (L's ids
 * ascending padded with -1, then U's), in no particular order.  *n_out is the number of
 * pairs; at most cap rows are written (call with cap 0 to size the buffer).
 * field and rows: host memory. */
msc_status msc_gradient_pairs(const float *field, int nx, int ny, int nz,
                              int64_t *rows, uint64_t cap, uint64_t *n_out);

/* Sec. 3.1: critical (unpaired) cells of a field: rows of 4 int64 vertex ids (ascending,
 * -1 padded) and their dimensions, in no particular order.  Host memory. */
msc_status msc_critical_cells(const float *field, int nx, int ny, int nz,
                              int64_t *rows, int32_t *dims, uint64_t cap, uint64_t *n_out);

/* Largest grid (in vertices) that msc_critical_cells_static accepts. */
#define MSC_STATIC_MAX_VERTICES (1u << 20)

/* Same result as msc_critical_cells, for callers that cannot allocate device memory: for
 * example a host application that hands this library a fixed memory budget through its
 * own allocator, or a code path that must not call cudaMalloc/cudaFree because those
 * calls can synchronize the device.  The paper has no counterpart to this entry point.
 *  - field (nx*ny*nz floats), rows (cap x 4 int64) and dims (cap int32) are DEVICE
 *    pointers on the current device, allocated and owned by the caller; host pointers are
 *    rejected with MSC_ERR_INVALID_ARG.  *n_out (host memory) receives the number of
 *    critical cells; at most cap rows are written, in no particular order.
 *  - Scratch space is a fixed static device array of MSC_STATIC_MAX_VERTICES 8-byte words
 *    plus a few counters (about 8 MiB), which every GPU that loads the library keeps until
 *    the process exits.  Grids larger than MSC_STATIC_MAX_VERTICES vertices are rejected
 *    with MSC_ERR_INVALID_ARG.  No device memory is allocated or freed by this call.
 *  - Every call looks up the device address of that array (cudaGetSymbolAddress) on the
 *    current device, queues its kernels on stream, then waits for that stream before it
 *    returns, on success and on every error path alike (so no call can be captured into a
 *    CUDA graph).
 *  - All calls share the one array (its counters are cleared at the start of each call):
 *    calls whose device work overlaps (other threads or streams) race and give wrong
 *    results.  stream: a cudaStream_t (NULL = the legacy default stream).
 *  - Device pointers of another device are rejected with MSC_ERR_INVALID_ARG before any
 *    kernel is launched.  On any status other than MSC_OK the contents of rows and dims
 *    are undefined. */
msc_status msc_critical_cells_static(const float *field, int nx, int ny, int nz, int64_t *rows, int32_t *dims,
                                     uint64_t cap, uint64_t *n_out, void *stream);

/* Bytes of the library's device memory pool on the current device that are allocated to
 * live buffers right now (cudaMemPoolAttrUsedMemCurrent); memory the pool keeps for reuse
 * is not counted.  Lets a caller check that a sequence of calls allocated nothing. */
msc_status msc_pool_used_bytes(uint64_t *used);

/* The tile autotuner of the dense 3D gradient.  The first dense pass of a grid shape on a
 * device (with the tile options 0) times every instantiated tile shape once on its input and
 * keeps the fastest for that (device, nx, ny, nz); every shape gives the same result.  This
 * reports, for the current device and a grid: *n = the number of shapes, shapes[3*i ..] the
 * anchors per block along x, y, z of shape i and ms[i] its time on the tuning pass (up to cap
 * shapes), chosen[0..2] the shape kept (all 0, and ms 0, if the grid was not tuned yet).
 * Any of chosen, shapes, ms may be NULL. */
msc_status msc_tile_report(int nx, int ny, int nz, int *chosen, int *shapes, float *ms, int cap, int *n);

/* Launch statistics accumulated on a handle since its creation or the last reset. */
msc_status msc_get_stats(msc_handle *h, msc_stats *out);
msc_status msc_reset_stats(msc_handle *h);

/* Bytes of device memory a handle of this grid holds while fixing (for admission). */
uint64_t msc_device_bytes(int nx, int ny, int nz);

/* Device memory that handles free stays in the library's memory pool on that device, so
 * that the next handle of a similar size reuses it without going back to the driver (a
 * server limits what the pool keeps to its memory budget).  Likewise the page-locked host
 * buffers of edit records that msc_free_edits gives back are kept (up to 8 GiB) for the
 * next record.  This call returns everything the pool of the current device holds unused
 * to the driver and frees the kept host buffers, after waiting for the device to finish its
 * work.  Handles and edit records that are still alive keep their memory. */
msc_status msc_release_cached_memory(void);

/* Fault injection for tests (not part of the method; off by default).  After `after`
 * further device allocations succeed, the next `count` device allocations of the library
 * fail as if the device were out of memory (the call that needed them returns MSC_ERR_OOM
 * and frees what it had allocated); later allocations succeed again.  The failure is made
 * on the host: no device call fails and the device is not touched.  count = 0 turns the
 * injection off.  Process-wide; returns the number of failures injected so far. */
uint64_t msc_inject_alloc_failures(uint64_t after, uint64_t count);

/* Walk limits for tests (not part of the method).  The saddle-saddle propagation of the
 * separatrix state (Sec. 4.4) keeps its pending triangles on a stack per warp in shared
 * memory (384 entries) and, in the incremental update, lets one thread walk up to 512 steps
 * before it hands the rest of its stack to a spill queue that a converged kernel drains.
 * warp_stack (1..384) and local_steps (>= 1) lower these limits for the next fixes so that
 * small fields take the spill paths; 0 for either restores its default.  Results do not
 * depend on the limits (every change is an atomic on a node word).  Process-wide; returns
 * MSC_ERR_INVALID_ARG for a warp_stack above 384. */
msc_status msc_set_walk_limits(uint32_t warp_stack, uint32_t local_steps);

/* Self-test of the bounded waits (not part of the method).  The persistent round kernel
 * separates its phases with a grid barrier whose wait gives up after 2 s of device time,
 * records MSC_ERR_DEVICE_TIMEOUT and ends the kernel, so that a block that never arrives
 * cannot hang the device.  This call launches that barrier in a kernel where one block waits
 * for another that never arrives, with a limit of timeout_ms (1..2000) milliseconds.  It
 * returns MSC_ERR_DEVICE_TIMEOUT when the wait gave up and reported it (the expected outcome;
 * the device stays usable), MSC_ERR_CUDA otherwise.  stream: a cudaStream_t (NULL = the
 * legacy default stream). */
msc_status msc_selftest_barrier(int timeout_ms, void *stream);

/* ---------------------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  The paper runs one field at a time;
 * this runtime admits fix jobs as they arrive and runs several at once on one GPU.
 *  - A job holds msc_device_bytes of its grid from admission to completion.  A queued job
 *    is admitted, first fit in arrival order, as soon as one of max_jobs slots is free and
 *    its bytes fit in what mem_budget has left.  A job that keeps being passed over by
 *    smaller ones (max_skips times) blocks admission until it fits.
 *  - Each slot is a host thread with its own non-blocking stream: it prepares the job's
 *    original (gradient of f, separatrix seeds), runs the whole fix loop with the job's
 *    state resident on the device, copies g out and frees the job's memory.  Slots run
 *    concurrently, so the rounds of different jobs overlap on the device.
 *  - Device memory comes from the device's default stream-ordered memory pool; the server
 *    sets that pool's release threshold to mem_budget, so freed job memory stays cached
 *    for the next job instead of going back to the driver.
 *  - A job's result equals that of msc_prepare_original + msc_fix on the same inputs.
 * --------------------------------------------------------------------------------------- */
typedef struct msc_server msc_server;

typedef struct {
    int max_jobs;          /* jobs on the device at once (slots), 1..64 */
    int max_skips;         /* admissions that may pass a waiting job before it blocks the
                              queue (0 = 16) */
    uint64_t mem_budget;   /* device bytes the admitted jobs may hold together; 0 = 90% of
                              the free device memory at creation */
    msc_options options;   /* tier, q_max, max_iters, exact_fallback, profile for every job;
                              stream is ignored (each slot has its own) */
} msc_server_config;

typedef struct {
    int32_t status;        /* msc_status of the job */
    int32_t slot;          /* slot that ran it */
    uint64_t bytes;        /* device bytes reserved at admission */
    double t_submit, t_start, t_end;   /* seconds since the server was created (steady clock) */
    float loop_ms;         /* device time of the fix loop */
    uint32_t reserved;
} msc_job_info;

/* Create a server on the current device.  cfg: NULL for defaults (8 slots, 90% of free
 * memory, default options).  Errors: MSC_ERR_INVALID_ARG for bad settings. */
msc_status msc_server_create(const msc_server_config *cfg, msc_server **out);

/* Queue one job and return at once with its ticket.  f, f_hat (nx*ny*nz floats, host or
 * device) and g_out (same size, host or device) stay owned by the caller and must remain
 * valid until msc_server_wait returns for this ticket.  Errors: MSC_ERR_INVALID_ARG (dims,
 * xi), MSC_ERR_OOM when the job alone exceeds mem_budget. */
msc_status msc_server_submit(msc_server *srv, const float *f, const float *f_hat, int nx, int ny, int nz, float xi,
                             float *g_out, uint64_t *ticket);

/* Block until the job ends, then release it from the server.  *out receives its edits
 * (free with msc_free_edits; NULL to discard) and *info its record (may be NULL).
 * Returns the job's status; MSC_ERR_INVALID_ARG for an unknown ticket. */
msc_status msc_server_wait(msc_server *srv, uint64_t ticket, msc_edits *out, msc_job_info *info);

/* Cancel a job.  A queued job is taken off the queue at once; a running job stops at the
 * next point where its fix loop returns to the host (between round launches), frees its
 * state and ends.  Either way msc_server_wait then returns MSC_ERR_CANCELLED for it (a
 * running job that finishes before it reaches such a point keeps its own status).  Returns
 * MSC_OK, or MSC_ERR_INVALID_ARG for an unknown ticket or a job that has already ended. */
msc_status msc_server_cancel(msc_server *srv, uint64_t ticket);

/* Finish the running jobs, cancel the queued ones and free the server.  No other call on
 * this server (submit, wait) may run concurrently with or after this one. */
void msc_server_destroy(msc_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* MSC_H */
