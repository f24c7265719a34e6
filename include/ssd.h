/*
 * ssd.h - C ABI of the GB300 sliding super point detector.
 *
 * Sliding super point detection from distributed edge routers (arXiv
 * 1803.11036): every router scans the <cip, oip> IPv4 pairs of each time slot
 * into its own reversible sliding estimator array (RSEA); at the end of a slot
 * the routers' arrays are merged and the sliding super points - hosts with at
 * least theta distinct opposite hosts within the last k slots (Def. 2-4) - are
 * regained through the reversible hash functions group (RHFG).
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers on the context's device; pointers
 *    marked "host or device" may be either (unified addressing). The caller
 *    owns every buffer it passes; the library owns contexts, sketches and the
 *    scratch memory a context allocates at creation.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Calls enqueue work on it and return without waiting unless they
 *    say otherwise. Work for one context must not run on two streams at once:
 *    a context holds one set of scratch buffers.
 *  - Every call returns SSD_OK (0) or a negative SSD_E* code; no exception or
 *    abort crosses the ABI. On SSD_EINVAL nothing was enqueued.
 *  - Packet pairs are uint32 pairs laid out (cip, oip), 8 bytes per packet,
 *    host-order IPv4 values (Sec. 3.1). A pair buffer must be 8-byte aligned.
 *  - A sketch is r rows x 2^q columns of sliding estimators, each eta = 2^log2_eta
 *    uint16 distance recorders, stored row-major: recorder j of estimator
 *    (row, col) is element ((row * 2^q) + col) * eta + j (Sec. 3.3).
 *  - Wherever recorders cross this ABI (ssd_sketch_export, ssd_sketch_import,
 *    ssd_regain_static, ssd_min_merge) they are the paper's distances: 0..65534
 *    slots since a pair last set the recorder, 65535 for never or for 65535 slots
 *    or more (Sec. 3.2). Inside a sketch the library stores each one as a stamp,
 *    the slot counter modulo 65535 when a pair last set it (0xFFFF for distance
 *    65535), next to the sketch's clock (its slot counter modulo 65535) in
 *    device memory: the advance of every recorder by one is then the clock's
 *    tick, and a slot writes only the recorders its pairs set (and, once in
 *    65535 slots, those whose distance reaches 65535). Distances are a pure
 *    function of the stamps and the clock, so every count, list and exported
 *    array is that of the paper's recorders. ssd_sketch_data exposes the stamps.
 */
#ifndef SSD_H
#define SSD_H

#include <stdint.h>

#if defined(__GNUC__)
#define SSD_API __attribute__((visibility("default")))
#else
#define SSD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define SSD_OK 0
#define SSD_EINVAL (-1)    /* bad argument or parameter set */
#define SSD_ENOMEM (-2)    /* device allocation failed */
#define SSD_ECAPACITY (-3) /* a capacity was exceeded; see ssd_stats */
#define SSD_ECUDA (-4)     /* a CUDA call failed; ssd_last_cuda_error() names it */
#define SSD_ETIMEOUT (-5)  /* reserved: a bounded device-side wait ran out */
#define SSD_ESTATE (-6)    /* sketches disagree on their slot, or belong to another context */

/* ------------------------------------------------------------------ flags */
/* Also require RHFG[0](cip) == he_0 of the tuple a host is regained from. The
 * paper does not make this check (Algorithm 4 extracts the host directly);
 * without it a tuple mixing several hosts' estimators can name a host that is
 * not there. Off by default. */
#define SSD_VERIFY_H0 1u
/* Do not prune partial candidate tuples by their union's R_k: run the candidate
 * levels literally (Algorithms 6-7). The list is identical either way; only the
 * candidate counts (and the work) differ. */
#define SSD_NO_PRUNE 2u
/* ssd_slot, one router: collect every chunk's touch bits on the side stream, as
 * for several routers, instead of inside the streaming kernel. Same result. */
#define SSD_SLOT_CHUNKED 4u
/* Eq. 2 as printed: RHFG[i](cip) = ((cip >> (i*delta)) XOR RHFG[0](cip)) mod 2^q.
 * By default the shift is (i-1)*delta, the only shift under which the stated
 * condition (r-2)*delta + q >= 32 puts every bit of cip in some window B(i)
 * (Eq. 3). With the printed shift no window holds bits 0..delta-1: a tuple
 * fixes bits delta..31 only, and the regain tries the 2^delta completions and
 * lists those whose RHFG[0] is he_0 (so the check of SSD_VERIFY_H0 is implied).
 * For comparing the two readings. */
#define SSD_RHFG_LITERAL 8u

#define SSD_MAX_R 8
#define SSD_MAX_ROUTERS 128

/* Detector parameters (Sec. 3.2-3.3, Sec. 5).
 *   eta = 2^log2_eta recorders per estimator, 5 <= log2_eta <= 15
 *   2^q columns, r rows, shift step delta:
 *       3 <= r <= SSD_MAX_R, 0 < delta < q <= 24, (r-2)*delta + q >= 32 (Eq. 2-3)
 *   k: window length in slots, 1 <= k <= 65534 (Sec. 3.2)
 *   theta: super point threshold (Def. 2), >= 1
 *   flags: SSD_VERIFY_H0 | SSD_NO_PRUNE | SSD_SLOT_CHUNKED | SSD_RHFG_LITERAL
 *   hse_capacity: hot estimators kept per row (0 = min(2^q, 65536))
 *   ctb_capacity: tuples per candidate tuple buffer (0 = 2^22)
 *   out_capacity: accepted tuples staged before the list is sorted (0 = 2^20)
 *   touch_chunk_bytes: touch bits per chunk of ssd_slot, kept in L2 (0 = 32 MiB)
 */
typedef struct ssd_params {
  uint32_t log2_eta;
  uint32_t q;
  uint32_t r;
  uint32_t delta;
  uint32_t k;
  uint32_t theta;
  uint32_t flags;
  uint32_t hse_capacity;
  uint64_t ctb_capacity;
  uint64_t out_capacity;
  uint64_t touch_chunk_bytes;
} ssd_params;

typedef struct ssd_ctx ssd_ctx;
typedef struct ssd_sketch ssd_sketch;

/* Counters of the last regain or slot close of a context. */
#define SSD_STATUS_HSE_OVERFLOW 1u  /* more hot estimators in a row than hse_capacity */
#define SSD_STATUS_CTB_OVERFLOW 2u  /* more candidate tuples than ctb_capacity */
#define SSD_STATUS_OUT_OVERFLOW 4u  /* more accepted tuples than out_capacity */
#define SSD_STATUS_LIST_OVERFLOW 8u /* more hosts than the caller's list capacity */
#define SSD_STATUS_INTERNAL 16u     /* an internal bound was broken: a library fault, the
                                       result of the call is not valid (never set by design;
                                       see also the SSD_DEBUG build) */
typedef struct ssd_stats {
  uint32_t status;           /* OR of SSD_STATUS_* */
  uint32_t threshold;        /* ceil(R^_k), R^_k = eta * (1 - exp(-theta/eta)) (Sec. 3.3) */
  uint64_t hot[SSD_MAX_R];   /* |HSE(i)|: hot estimators of row i, all of them */
  uint64_t level[SSD_MAX_R]; /* candidates covering rows 0..i: level[1] pairs, level[2] the
                                CT_2 triples of Algorithm 6, level[i>2] Algorithm 7's tuples */
  uint64_t raw;              /* full tuples accepted by the final test, before dedupe */
  uint64_t n_out;            /* hosts in the sliding super point list */
} ssd_stats;

/* Validate a parameter set (host only, no GPU needed). SSD_OK or SSD_EINVAL. */
SSD_API int ssd_params_check(const ssd_params* p);

/* ceil(eta * (1 - exp(-theta/eta))), the integer R_k at which an estimator is
 * hot (Sec. 3.3), computed in double on the host (no GPU needed). SSD_EINVAL if
 * the real threshold lies within 1e-9 of an integer. */
SSD_API int ssd_threshold(const ssd_params* p, uint32_t* thr);

/* Create a context on `device`. `tables` (host) holds 2048 uint32 words: the
 * simple-tabulation tables of H1 (words 0..1023: T0..T3, 256 each; Sec. 3.2)
 * followed by those of RHFG[0] (words 1024..2047; Sec. 3.3). The context
 * copies them, computes the threshold and allocates its scratch (hot-estimator
 * pools, candidate tuple buffers CTB_1/CTB_2 of Sec. 4.2, the list staging
 * buffer). Returns SSD_EINVAL, SSD_ENOMEM or SSD_ECUDA on failure (*out = NULL). */
SSD_API int ssd_create(const ssd_params* p, const uint32_t* tables, int device, ssd_ctx** out);
SSD_API void ssd_destroy(ssd_ctx* ctx);

/* One RSEA (a router's, or the global one), every recorder set to 65535
 * (Sec. 3.2), slot counter 0. Synchronous. A sketch may be destroyed before or
 * after its context, but no call may use it once the context is gone. */
SSD_API int ssd_sketch_create(ssd_ctx* ctx, ssd_sketch** out);
SSD_API void ssd_sketch_destroy(ssd_sketch* s);
/* Bytes of one RSEA: r * 2^q * eta * 2. */
SSD_API uint64_t ssd_sketch_bytes(const ssd_ctx* ctx);
/* Slots the sketch has advanced since creation or import. */
SSD_API int ssd_sketch_slot(const ssd_sketch* s, uint64_t* slot);
/* Set the host's slot counter (host bookkeeping only, no GPU work): after
 * replaying a captured slot the caller advances the counters the replay cannot.
 * The device clock the stamps refer to is moved on by the advancing calls
 * themselves (and by their replays), never by this call. */
SSD_API int ssd_sketch_set_slot(ssd_sketch* s, uint64_t slot);
/* What a sketch counts (its view). Sec. 3.1 defines sliding super points for
 * the hosts of CNet, the first field of each pair, and obtains those of ONet by
 * exchanging the roles of the two networks; Sec. 6 scales to bigger networks by
 * keeping several RSEAs, each regaining one group of hosts split by their IP
 * addresses.
 *   side: SSD_SIDE_CNET - hosts are the first field of a pair, opposite hosts
 *         the second (the default); SSD_SIDE_ONET - the other way round;
 *   group_bits (0..SSD_MAX_GROUP_BITS), group (< 2^group_bits): the sketch takes
 *         only pairs whose host has `group` as its top group_bits bits; every
 *         scan skips the others, and a regain of the sketch lists only hosts of
 *         the group (a tuple naming a host of another group is rejected: no pair
 *         of that host reached the sketch). group_bits = 0: every host.
 * A view is set before the sketch's first scan (SSD_ESTATE once it has advanced
 * a slot; scans made earlier in slot 0 counted under the old view). Calls that
 * combine sketches (ssd_merge, ssd_close_slot, ssd_slot) need one view for all
 * of them (SSD_EINVAL) and the global sketch takes it; ssd_scan_batch may mix
 * views, so one launch can scan the same pairs for both sides (bidirectional
 * detection) or for every group. */
#define SSD_SIDE_CNET 0u
#define SSD_SIDE_ONET 1u
#define SSD_MAX_GROUP_BITS 16
SSD_API int ssd_sketch_set_view(ssd_sketch* s, uint32_t side, uint32_t group_bits, uint32_t group);
SSD_API int ssd_sketch_view(const ssd_sketch* s, uint32_t* side, uint32_t* group_bits, uint32_t* group);
/* Occupancy of a sketch (diagnostics, not on the slot path): rk_sum[i] (host,
 * r entries) receives the sum over row i's 2^q estimators of R_k, the recorders
 * below k (Sec. 3.2). A row's mean R_k gives through Eq. 1 the distinct opposite
 * hosts its columns hold, the realised column load. Reads the whole RSEA once
 * and waits for `stream`. */
SSD_API int ssd_sketch_occupancy(const ssd_sketch* s, uint64_t* rk_sum, void* stream);
/* The device address of the sketch's stored recorders (ssd_sketch_bytes bytes,
 * laid out as described at the top of this file, in the stamp form: not
 * distances), owned by the library and valid until the sketch is destroyed; the
 * sketch's clock (uint32, its slot counter modulo 65535) follows them. For
 * inspecting or checkpointing the raw state in place; to move recorders between
 * GPUs as distances, export them to device memory (ssd_sketch_export) and import
 * them on the other side. The caller orders such access against the context's
 * stream. */
SSD_API int ssd_sketch_data(const ssd_sketch* s, uint16_t** d_recorders);
/* The reduction of Algorithm 5 when the routers' RSEAs are spread over several
 * GPUs (the paper ships every monitor server's RSEA to one server, Sec. 4):
 * d_out[x] = min over j < n of d_in[j][x] for x < count, the elementwise
 * minimum of the union reading (as ssd_merge). Each GPU folds the slices of
 * one recorder range that it received from the others; collective libraries
 * offer no 16-bit minimum, so they move the bytes and this call reduces them.
 * d_in is a host array of n (1..SSD_MAX_ROUTERS) device pointers; d_out and
 * every d_in[j] must be 16-byte aligned on the context's device (SSD_EINVAL
 * otherwise; with count = 0 nothing is read). d_out may be one of the inputs.
 * Asynchronous on `stream`. */
SSD_API int ssd_min_merge(ssd_ctx* ctx, uint16_t* d_out, const uint16_t* const* d_in, int n, uint64_t count,
                          void* stream);
/* Write the distances (Sec. 3.2) of `count` recorders starting at recorder
 * `first` to dst (host or device; device memory is written by a kernel, host
 * memory through a staging buffer the context allocates on first use, up to
 * 32 MiB). Waits for `stream` before returning. Checkpointing a sketch is
 * export + ssd_sketch_slot; resuming is import. */
SSD_API int ssd_sketch_export(const ssd_sketch* s, uint64_t first, uint64_t count, uint16_t* dst, void* stream);
/* Overwrite the whole sketch from the distances in src (host or device;
 * ssd_sketch_bytes bytes) and set its slot counter (and clock) to `slot`. Waits
 * for `stream` before returning. */
SSD_API int ssd_sketch_import(ssd_sketch* s, const uint16_t* src, uint64_t slot, void* stream);

/* Algorithm 2 for every pair of d_pairs[0 .. 2*n_pairs): DRidx = H1(oip); for
 * each row i the recorder DRidx of estimator RSEA[i, RHFG[i](cip)] is set to 0,
 * with RHFG[i](cip) = ((cip >> (i-1)*delta) XOR RHFG[0](cip)) mod 2^q for
 * i >= 1 (Eq. 2). Order-free and idempotent (Sec. 4.1). n_pairs may be 0. */
SSD_API int ssd_scan(ssd_sketch* s, const uint32_t* d_pairs, uint64_t n_pairs, void* stream);

/* Algorithm 2 on pairs held in HOST memory (pinned or pageable): the pairs go
 * over the host link into a context-owned device buffer of `alpha` pairs
 * (Sec. 4.1; two such buffers, allocated on the first call, 2^22 pairs each)
 * and each filled buffer is scanned while the next one is copied. Copies run
 * on an internal stream ordered against `stream`; scans run on `stream`. With
 * pinned memory the call returns before the copies finish: keep h_pairs
 * unchanged until `stream` has reached this point. The first call on a
 * context allocates; make it before any stream capture. */
SSD_API int ssd_scan_host(ssd_sketch* s, const uint32_t* h_pairs, uint64_t n_pairs, void* stream);

/* Algorithm 2 for n routers in one launch: router j scans d_pairs[j] (n_pairs[j]
 * packets) into sketches[j]. sketches, d_pairs and n_pairs are host arrays of n
 * entries, n <= SSD_MAX_ROUTERS; the sketches share one context (an entry may
 * repeat). Same result as n calls of ssd_scan. */
SSD_API int ssd_scan_batch(ssd_sketch* const* sketches, const uint32_t* const* d_pairs, const uint64_t* n_pairs,
                   int n, void* stream);

/* Window advance (Sec. 3.2, Sec. 4.3): every recorder below 65535 of each of
 * the n sketches grows by one; each sketch's slot counter grows by one. (One
 * read pass stores 0xFFFF into the recorders whose distance reaches 65535, then
 * the sketches' clocks tick; no other recorder is written.) */
SSD_API int ssd_advance(ssd_sketch* const* sketches, int n, void* stream);

/* Algorithm 5: global[x] = UnionSE of routers[0..n)[x] for every recorder x,
 * read as the elementwise minimum (the union of "distance to the nearest slot";
 * Algorithm 1 prints a maximum, which would keep only recorders every router
 * saw). All routers must be at the same slot (else SSD_ESTATE); the global
 * sketch takes that slot. `global` must not be one of the routers. */
SSD_API int ssd_merge(ssd_sketch* const* routers, int n, ssd_sketch* global, void* stream);

/* Regain the sliding super points of a (global) sketch (Sec. 3.3, Sec. 4.2):
 * hot estimators (R_k >= threshold, R_k = recorders below k), candidate tuples
 * row by row with the overlap test between B(i-1) and B(i), B(j) = he_0 XOR
 * he_j (Algorithms 6-7), and the final test R_k(UnionSE of the tuple) >=
 * threshold with UnionSE the elementwise maximum (Algorithm 1), after which the
 * host is the 32-bit value whose q-bit windows are B(1..r-1) (a tuple naming a
 * bit beyond bit 31 yields none). The list is ascending and duplicate-free; a
 * host regained from several tuples gets the largest R_k.
 * Writes up to `cap` hosts to d_ips and their R_k to d_rk (device) and the list
 * size to *n_out (host). Waits for `stream`. Returns SSD_ECAPACITY when the
 * list is longer than cap (*n_out = the full size, nothing written) or when an
 * internal capacity overflowed (see ssd_stats_get). */
SSD_API int ssd_regain(ssd_ctx* ctx, const ssd_sketch* global, uint32_t* d_ips, uint32_t* d_rk, uint64_t cap,
               uint64_t* n_out, void* stream);

/* The regain of ssd_regain for callers that cannot allocate device memory: a
 * process whose device memory is already claimed by another framework's
 * caching allocator, or a datapath that must not pay cudaMalloc's implicit
 * device synchronisation. It needs no context and allocates nothing: its
 * scratch is one fixed 32 MiB device array inside the library, which every GPU
 * that loads the library holds until the process exits. (The paper has no
 * counterpart; this is a deployment variant of the same computation.)
 *   p: the parameter set (its capacity fields are ignored: the array decides
 *      them, at most 4096 hot estimators per row);
 *   side, group_bits, group: the view of the sketch the recorders come from
 *      (ssd_sketch_view; checked as ssd_sketch_set_view checks them). With
 *      group_bits > 0 the list holds only hosts of `group`, as in ssd_regain;
 *   d_tables: the 2048 hash-table words of ssd_create, in device memory;
 *   d_recorders: a whole RSEA (ssd_sketch_bytes bytes, 16-byte aligned) in
 *      device memory on the current device;
 *   d_ips, d_rk, cap, *n_out: as in ssd_regain.
 * Runs on the caller's current device. Every call looks up the array's device
 * address on that device (cudaGetSymbolAddress) and waits for `stream` before
 * returning (synchronous). Returns SSD_ECAPACITY when the parameter set needs
 * more scratch than the array holds (r * 2^q four-byte entries must stay under
 * 16 MiB: q <= 19 at r = 5) or when a capacity overflowed. Every call shares
 * the one array and leaves its contents behind (the counters are cleared at
 * the start of each call); calls that overlap on the GPU race and must be
 * serialised by the caller. */
SSD_API int ssd_regain_static(const ssd_params* p, uint32_t side, uint32_t group_bits, uint32_t group,
                              const uint32_t* d_tables, const uint16_t* d_recorders, uint32_t* d_ips,
                              uint32_t* d_rk, uint64_t cap, uint64_t* n_out, void* stream);

/* End of slot for n routers, fully asynchronous and free of host
 * synchronisation (it can be captured in a CUDA graph): one streaming pass
 * merges the routers (Algorithm 5, min reading), writes the merged RSEA to
 * `global` when it is not NULL, finds the hot estimators of the merged RSEA and
 * then advances every router's recorders (Sec. 4.3); the candidate levels, final
 * test and list follow as in ssd_regain. The list size goes to *d_n_out (device
 * uint64); the list itself to d_ips/d_rk when it fits `cap`. Status and
 * counters are read afterwards with ssd_stats_get. Routers must share one slot
 * (SSD_ESTATE); each advances by one slot, `global` takes the merged slot. */
SSD_API int ssd_close_slot(ssd_ctx* ctx, ssd_sketch* const* routers, int n, ssd_sketch* global, uint32_t* d_ips,
                   uint32_t* d_rk, uint64_t cap, uint64_t* d_n_out, void* stream);

/* Tracing: when set, ssd_close_slot and ssd_regain record ev_start just before
 * their streaming pass, ev_pass after the streaming pass (merge / hot extraction
 * / advance) and ev_end after the list is written, on their stream. The events
 * are cudaEvent_t passed as void*, created by the caller; NULLs switch tracing
 * off. */
SSD_API int ssd_set_trace(ssd_ctx* ctx, void* ev_start, void* ev_pass, void* ev_end);

/* A whole slot for n routers in one call: Algorithm 2 for every router's pairs
 * followed by the end of slot of ssd_close_slot - the same result as
 * ssd_scan_batch(routers, d_pairs, n_pairs, n) then ssd_close_slot(...), with
 * the same arguments and the same asynchrony (no host synchronisation).
 * The recorders are not written by the scan: the estimators are taken in
 * chunks whose touch bits (one bit per recorder and router, touch_chunk_bytes
 * per chunk, double-buffered) stay in L2; a side stream collects the touches of
 * chunk c+1 while the streaming pass applies those of chunk c (recorder := 0,
 * Sec. 4.1), merges, extracts the hot estimators and advances. Every recorder
 * is read once per slot; only the vectors holding a touched (or expiring)
 * recorder are written, and no random DRAM write remains. When the routers'
 * touch bits would need more than 16 chunks the call runs ssd_scan_batch and
 * ssd_close_slot instead (same result).
 * One router with eta >= 256 (unless SSD_SLOT_CHUNKED) uses one stream: the
 * pairs are hashed once per slot (into per-chunk touch lists, or into packed
 * hashes with ssd_tuning's collect_touches = 1) and chunk 0's bits set by that
 * launch or the next; then the streaming kernel of each chunk, between
 * estimators, sets the next chunk's bits, so the collection fills the memory
 * stalls of the stream; up to 32 chunks. */
SSD_API int ssd_slot(ssd_ctx* ctx, ssd_sketch* const* routers, const uint32_t* const* d_pairs,
                     const uint64_t* n_pairs, int n, ssd_sketch* global, uint32_t* d_ips, uint32_t* d_rk,
                     uint64_t cap, uint64_t* d_n_out, void* stream);

/* ssd_slot on pairs held in HOST memory (pinned for overlap): each router's
 * pairs are copied on an internal copy stream into one of two context-owned
 * device staging areas (the alpha-pair buffer of Sec. 4.1, sized to the slot),
 * then ssd_slot runs on `stream`. The copy of one call overlaps the slots still
 * running from earlier calls. With pinned memory the call returns before the
 * copies finish: keep h_pairs unchanged until `stream` has passed this call. A
 * slot larger than any earlier one (re)allocates the staging areas, waiting for
 * the context's work first; make the first call before any stream capture. */
SSD_API int ssd_slot_host(ssd_ctx* ctx, ssd_sketch* const* routers, const uint32_t* const* h_pairs,
                          const uint64_t* n_pairs, int n, ssd_sketch* global, uint32_t* d_ips, uint32_t* d_rk,
                          uint64_t cap, uint64_t* d_n_out, void* stream);

/* Allocate now what ssd_slot and ssd_slot_host would otherwise allocate on a
 * first call with up to max_pairs pairs in the slot (summed over its routers):
 * the pre-hashed pairs and the host staging areas. Later calls with at most
 * that many pairs allocate nothing, so ssd_slot can be captured in a CUDA graph
 * (stream capture cannot allocate). Waits for the device. */
SSD_API int ssd_reserve(ssd_ctx* ctx, uint64_t max_pairs);

/* Launch configuration of a context's kernels. The paper has no counterpart:
 * these choices set only how the work of Algorithms 2 and 5 and of the
 * streaming pass (Sec. 4.3) is spread over the GPU. No value changes a
 * recorder, a list or a counter. Defaults: touch_chunk_bytes of the params, 0, 8,
 * 4, 8, 0, 0, 0.
 *   touch_chunk_bytes: touch bits of one chunk of ssd_slot (64 KiB .. 1 GiB,
 *       rounded up to 256 B; chunk sizes are powers of two that fit it);
 *   stream_blocks_per_sm: resident blocks per SM of the streaming and chunk
 *       kernels (0 = as many as fit, else at most this many, 1..8);
 *   scan_blocks_per_sm: the scan, touch and pre-hash kernels launch at most
 *       SMs x this many blocks (1..32);
 *   scan_unroll: 16-byte pair vectors one thread loads before hashing them
 *       (items per thread per step: 1, 2, 4 or 8);
 *   merge_group: routers whose recorders one lane loads before it stores any
 *       of them in the multi-router streaming pass (the merge tile: 2, 4 or 8);
 *   combine_touches: how touches that land on one 32-bit word of the touch
 *       bits are combined. 0 = one atomic per touch; 1 = the lanes of a warp
 *       whose bits fall into one word OR them together (__match_any_sync) and
 *       issue one atomic; 2 = the word is read from L2 first and the atomic is
 *       skipped when the bit is already set, which removes the repeats of a
 *       source that sends many packets to few peers;
 *   collect_touches: where the chunk launches of a one-router ssd_slot find the
 *       next chunk's touches. 0 = per-chunk touch lists: one launch hashes every
 *       pair once per slot, sets chunk 0's touch bits and writes the bit index
 *       of every other touch into its chunk's list (4 bytes per touch), so each
 *       chunk launch reads only its own touches; 1 = the slot's pairs, hashed
 *       once into (RHFG[0], H1) words, are re-read by every chunk launch;
 *   pair_level: how the pair level of the regain (HSE(0) x HSE(1), Sec. 4.2)
 *       computes the R_k of each pair's union. 0 = on the tensor cores, where it
 *       applies (eta a multiple of 128, pruning on): the popcounts of the ANDed
 *       "recorder < k" bitmaps are one matrix product of the bitmaps read as
 *       0/1 vectors, computed exactly as an fp8 GEMM with f32 sums; 1 = AND and
 *       popcount on the CUDA cores. */
typedef struct ssd_tuning {
  uint64_t touch_chunk_bytes;
  uint32_t stream_blocks_per_sm;
  uint32_t scan_blocks_per_sm;
  uint32_t scan_unroll;
  uint32_t merge_group;
  uint32_t combine_touches;
  uint32_t collect_touches;
  uint32_t pair_level;
  uint32_t reserved; /* must be 0 */
} ssd_tuning;

/* The context's current launch configuration (host only). */
SSD_API int ssd_tuning_get(const ssd_ctx* ctx, ssd_tuning* out);
/* Replace the launch configuration. SSD_EINVAL (nothing changed) for a value
 * outside the ranges above. A new touch_chunk_bytes reallocates the two touch
 * buffers after waiting for the device (make the call before any stream
 * capture; SSD_ENOMEM leaves the old configuration). */
SSD_API int ssd_tuning_set(ssd_ctx* ctx, const ssd_tuning* t);
/* Pick the launch configuration by measurement: run ssd_slot on the n routers
 * (and `global` when not NULL) with the given pairs - one representative slot,
 * device memory, as in ssd_slot - once per candidate value of one field at a
 * time, the others held at the best so far (two sweeps over the fields), `reps`
 * timed slots per candidate (1..16, the median counts) after one untimed one.
 * The fastest configuration is set on the context and written to *out (when
 * not NULL). The routers and `global` must not have run a slot yet (slot 0,
 * else SSD_ESTATE) and are returned to their initial state afterwards: every
 * recorder 65535, slot 0 (recorders scanned before the call are lost). Waits
 * for the device; not for use inside a stream capture. */
SSD_API int ssd_autotune(ssd_ctx* ctx, ssd_sketch* const* routers, const uint32_t* const* d_pairs,
                         const uint64_t* n_pairs, int n, ssd_sketch* global, int reps, ssd_tuning* out,
                         void* stream);

/* A counter the context increments whenever it frees or replaces a device
 * buffer that work captured in a CUDA graph may reference: the touch-bit buffers
 * (ssd_tuning_set with a new touch_chunk_bytes, ssd_autotune), the pre-hashed
 * pairs and the host staging areas (ssd_reserve, or an ssd_slot / ssd_slot_host
 * with a larger slot than any before). A graph captured at epoch e may be
 * replayed only while the epoch is still e. Host only; 0 for NULL. */
SSD_API uint64_t ssd_buffer_epoch(const ssd_ctx* ctx);

/* Counters of the context's last regain or close (waits for `stream`). */
SSD_API int ssd_stats_get(ssd_ctx* ctx, ssd_stats* out, void* stream);

/* Kernels this context has launched so far. */
SSD_API uint64_t ssd_launch_count(const ssd_ctx* ctx);

/* Message for an SSD_E* code (static storage). */
SSD_API const char* ssd_strerror(int code);
/* The last CUDA error seen by this thread inside the library, or "". */
SSD_API const char* ssd_last_cuda_error(void);
/* ABI version, major * 100 + minor. */
SSD_API int ssd_version(void);
/* How the library was built: SSD_BUILD_DEBUG when it is the debug build, whose
 * kernels check their indices against their bounds (a recorder inside its
 * estimator, a column inside its row, a touch bit inside its buffer, a pool,
 * bucket or candidate index inside its capacity), skip an access that breaks
 * one and report it as SSD_STATUS_INTERNAL in ssd_stats_get, which also checks
 * guard words around the candidate tuple buffers. The release build returns 0. */
#define SSD_BUILD_DEBUG 1
SSD_API int ssd_build_flags(void);

#ifdef __cplusplus
}
#endif

#endif /* SSD_H */
