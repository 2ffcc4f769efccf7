/*
 * gs_serve.h -- C ABI of the continuous-batching serving runtime around the zero-shot fitting
 * step of gs_api.h ("Physics-Driven 3D Gaussian Rendering for Zero-Shot MRI
 * Super-Resolution": Sec. 3.3 fits one Gaussian cloud per scan with the forward model of
 * Eq. 3-4 and the gradients of Eq. 5-6; Sec. 4.2 renders a fitted cloud on an arbitrary grid).
 * The paper fits one scan at a time and has no serving counterpart: this layer runs many
 * scans' fits and re-renders on one GPU at once.
 *
 * Model
 *   - The server owns one device arena of hbm_budget bytes, allocated at creation; all
 *     per-request device state (parameters, Adam moments, volumes, brick bins, workspace)
 *     is carved from it by a host-side best-fit allocator (gs_arena below). Admission is by
 *     that budget: a request is admitted when its state fits in the arena and fewer than
 *     max_active requests are resident.
 *   - Requests wait in arrival order. The oldest waiting request may be overtaken by later
 *     requests that fit when it does not, at most max_bypass times; then admission waits for
 *     it.
 *   - Each resident request owns one CUDA stream. A fit request advances in chunks of
 *     chunk_steps gs_fit_step calls (one replay of a graph captured at admission, or eager
 *     calls); the chunks of all resident requests run concurrently, and a request joins or
 *     leaves the resident set between chunks (continuous batching). A render request bins
 *     its cloud on its own grid and renders I (Eq. 3).
 *   - Outputs (fitted clouds, rendered volumes) outlive their request's residency until
 *     gs_server_release; they are placed at the top of the arena and transient state at the
 *     bottom, so finished outputs do not split the free space.
 *   - Pair capacity starts at pairs_per_gauss per Gaussian. A fitting step whose binning
 *     overflows is a no-op (gs_fit_step leaves the parameters, moments and step counter
 *     unchanged); the server reads the count needed after the chunk, grows the bins and goes
 *     on. Results therefore do not depend on capacity, chunking or what else is resident:
 *     in deterministic mode a request's output is bit-identical alone or in any mix.
 *   - Times are seconds on the server clock (a monotonic host clock started at creation). A
 *     request's completion time is the poll at which its last chunk was seen finished.
 *
 * Threading: the calls on one server must not overlap (one host thread drives it). All
 * device work is issued on the device that was current at gs_server_create; the entry
 * points make it current for their duration and restore the caller's device.
 */
#ifndef GS_SERVE_H
#define GS_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "gs_api.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ host-side allocator */

/* Best-fit allocator over a caller-provided address range (host bookkeeping only: it never
 * touches the memory, so the range may be device memory). Blocks are 256-byte aligned and
 * their sizes rounded up to 256 bytes; freed neighbours coalesce. */
typedef struct gs_arena gs_arena;

/* base: 256-byte aligned start of the range (not dereferenced); bytes: its length.
 * GS_ERR_INVALID_ARG on a null base or out pointer, or a misaligned base. */
gs_status gs_arena_create(void* base, size_t bytes, gs_arena** out);

/* *out = the lowest-addressed of the smallest holes of at least `bytes` (rounded up).
 * GS_ERR_CAPACITY (and *out = NULL) when no hole is large enough; bytes == 0 is invalid. */
gs_status gs_arena_alloc(gs_arena* a, size_t bytes, void** out);

/* Like gs_arena_alloc but from the top of the range: the block ends at the end of the
 * highest-addressed hole that can hold it. Long-lived blocks taken from the top and
 * short-lived ones from the bottom keep the free space in one piece. */
gs_status gs_arena_alloc_top(gs_arena* a, size_t bytes, void** out);

/* Return a block obtained from gs_arena_alloc or gs_arena_alloc_top. GS_ERR_INVALID_ARG if p
 * is not a live block. */
gs_status gs_arena_free(gs_arena* a, void* p);

/* Bytes in live blocks, their high-water mark, the largest hole, and the live block count.
 * Any output pointer may be NULL. */
gs_status gs_arena_stats(const gs_arena* a, size_t* used, size_t* peak, size_t* largest_free,
                         int64_t* n_live);

void gs_arena_destroy(gs_arena* a);

/* ------------------------------------------------------------------ server */

typedef struct gs_server gs_server;

typedef struct {
    size_t hbm_budget;      /* bytes of the device arena allocated at creation */
    int32_t max_active;     /* resident requests at once, one CUDA stream each: 1..64 */
    int32_t chunk_steps;    /* fitting steps per chunk: >= 1 */
    int32_t use_graphs;     /* 1: a chunk is one replay of a graph of chunk_steps steps */
    int32_t max_bypass;     /* >= 0: overtakes allowed past the oldest waiting request */
    float pairs_per_gauss;  /* initial pair capacity per Gaussian (> 0) */
    gs_config cfg;          /* rendering options for every request (gs_api.h) */
    gs_adam adam;           /* optimiser of every fit request */
} gs_server_config;

#define GS_REQ_FIT 0    /* fit a cloud to an LR scan through the z slice profile (L1, Adam) */
#define GS_REQ_RENDER 1 /* render a cloud on a grid: I of Eq. 3 */

#define GS_REQ_PENDING 0
#define GS_REQ_ACTIVE 1
#define GS_REQ_DONE 2
#define GS_REQ_FAILED 3

/* One request. Device inputs stay owned by the caller and must hold their values, with the
 * work that produced them finished, from gs_server_submit until the request leaves
 * GS_REQ_PENDING (they are copied into the arena at admission).
 *   kind: GS_REQ_FIT or GS_REQ_RENDER.
 *   grid: fit: the HR grid the cloud is rendered on; render: the output grid.
 *   lr_model: fit: GS_LR_ZBOX (slice factor s; lr_target has grid.nz / s slices) or
 *           GS_LR_TRILINEAR (lr_target is [lr_nz, lr_ny, lr_nx], the trilinear resize of the
 *           HR grid's field of view).
 *   s: fit with GS_LR_ZBOX: slice factor.
 *   iters: fit: number of fitting steps (>= 1).
 *   n_gauss: Gaussians in the cloud (>= 1); for a render of a fit's result, that fit's count.
 *   params: device float [n_gauss, 12]: fit: the initial cloud; render: the cloud to render
 *           (unused when source >= 0).
 *   lr_target: fit: device float of the LR shape.
 *   source: render: id of a fit request of this server whose fitted cloud is rendered (the
 *           render waits for it), or -1.
 *   arrival_s: the request is not admitted before this server-clock time. */
typedef struct {
    int32_t kind;
    gs_grid grid;
    int32_t s;
    int32_t iters;
    int64_t n_gauss;
    const float* params;
    const float* lr_target;
    int64_t source;
    double arrival_s;
    int32_t lr_model;
    int32_t lr_nx, lr_ny, lr_nz;
} gs_request;

/* State of one request.
 *   output: device, valid from GS_REQ_DONE until gs_server_release: fit: the fitted cloud
 *           [n_gauss, 12]; render: the volume I [nz, ny, nx]. NULL otherwise.
 *   loss: fit: L1 loss of the last step's forward pass.
 *   status_bits: OR of the GS_STATUS_* words seen (GS_STATUS_CAPACITY when the bins grew).
 *   capacity: the request's pair capacity now; grows: times it grew.
 *   bytes: arena bytes the request holds now. */
typedef struct {
    int32_t state;
    gs_status error;
    int32_t status_bits;
    int32_t steps_done;
    int64_t capacity;
    int32_t grows;
    int32_t chunks;
    float loss;
    double arrival_s, admit_s, done_s;
    const void* output;
    size_t bytes;
} gs_result;

typedef struct {
    double now_s;
    int32_t n_pending, n_active, n_done, n_failed;
    size_t arena_bytes, used_bytes, peak_bytes;
    int64_t chunks_launched, graphs_captured, grows;
} gs_server_stats;

/* Arena bytes a request needs at admission under cfg (host-only; 0 if the request is
 * invalid). A render of a fit's result needs its own n_gauss filled in. */
size_t gs_server_request_bytes(const gs_server_config* cfg, const gs_request* req);

/* Allocate the arena and max_active streams on the current device. GS_ERR_INVALID_ARG on a
 * bad configuration, GS_ERR_CUDA if the allocation fails. */
gs_status gs_server_create(const gs_server_config* cfg, gs_server** out);

/* Queue a request; *id receives its id (ids count from 0 in submission order).
 * GS_ERR_INVALID_ARG on an invalid request or unknown source; GS_ERR_CAPACITY if it could
 * never fit in the arena. */
gs_status gs_server_submit(gs_server* sv, const gs_request* req, int64_t* id);

/* One scheduling pass without blocking: retire finished chunks (growing bins where a chunk
 * overflowed), admit what fits, and launch the next chunk of every idle resident request.
 * *n_unfinished (may be NULL) = requests not yet DONE or FAILED. Returns GS_ERR_CAPACITY when
 * no request is resident and requests that have arrived do not fit beside the outputs the
 * arena still holds (release some; nothing else can make room). */
gs_status gs_server_poll(gs_server* sv, int32_t* n_unfinished);

/* Poll until every submitted request is DONE or FAILED, sleeping poll_us microseconds
 * between passes that change nothing. GS_ERR_TIMEOUT after timeout_s seconds, GS_ERR_CAPACITY
 * as gs_server_poll (requests keep their state; a later call continues). */
gs_status gs_server_run(gs_server* sv, double timeout_s, int32_t poll_us);

gs_status gs_server_result(const gs_server* sv, int64_t id, gs_result* out);

/* Free a finished request's output. GS_ERR_INVALID_ARG if it is not DONE or FAILED, or a
 * render request that is not finished still reads it. */
gs_status gs_server_release(gs_server* sv, int64_t id);

gs_status gs_server_stats_read(const gs_server* sv, gs_server_stats* out);

/* Wait for all device work, then free the arena, streams, graphs and events. */
void gs_server_destroy(gs_server* sv);

#ifdef __cplusplus
}
#endif

#endif /* GS_SERVE_H */
