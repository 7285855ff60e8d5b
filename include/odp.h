/*
 * odp.h -- C ABI of libodp, a B300 (sm_103a) implementation of the
 * data-parallel hot path of "Dynamic Detection of Inefficient Data Mapping
 * Patterns in Heterogeneous OpenMP Applications" (PPoPP '26):
 *
 *   1. content fingerprinting of mapped/transferred buffers (the paper, Sec. 5
 *      and 5.1, keeps a hash of the data of every transfer and assumes it
 *      collision-free; the hash here is the project-defined FP128 v1);
 *   2. detection over the mapping-event log of the patterns of Sec. 4
 *      (duplicate transfers, round trips, repeated allocations, unused
 *      allocations, unused transfers) with Algorithms 1-5 of Sec. 5, plus the
 *      wasted-time estimate of Sec. 7.6.
 *
 * Conventions for every call:
 *   - All pointers named "device" must be device memory of the current CUDA
 *     device (or managed memory); "host" pointers are ordinary host memory.
 *   - Calls are asynchronous on `stream` unless stated otherwise.  The caller
 *     keeps inputs and outputs alive and unmodified until the stream work
 *     completes.
 *   - The return value is a synchronous status (ODP_OK or a negative error);
 *     errors detected on the device are written to a device status word.
 *   - No C++ exception crosses this interface; kernels never trap.
 *   - Scratch memory comes from the allocator installed with
 *     odp_set_allocator (default: cudaMallocAsync on the call's stream) and is
 *     cached per (device, stream) between calls.
 */
#ifndef ODP_H
#define ODP_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */

enum {
    ODP_OK = 0,
    ODP_WARN_TRUNCATED = 1,     /* findings or site rows exceeded capacity  */
    ODP_ERR_INVALID_ARG = -1,   /* null pointer with n > 0, bad sizes       */
    ODP_ERR_CUDA = -2,          /* a CUDA runtime call failed               */
    ODP_ERR_OOM = -3,           /* the allocator returned null              */
    ODP_ERR_TIMEOUT = -4,       /* a bounded device-side wait ran out       */
    ODP_ERR_MALFORMED = -5,     /* an event record failed validation        */
    ODP_ERR_UNSORTED = -6,      /* event start times decrease               */
    ODP_ERR_UNSUPPORTED = -7,   /* input outside the implemented limits     */
    ODP_ERR_MISMATCH = -8       /* autotune: schedules disagreed (a bug)    */
};

/* Human-readable name of a status code (static string, never null). */
const char* odp_status_string(int status);

/* ----------------------------------------------------------- fingerprint */

/* 128-bit fingerprint: lo = bits 0..63, hi = bits 64..127. */
typedef struct odp_fp128 {
    uint64_t lo, hi;
} odp_fp128;

/*
 * odp_fingerprint -- FP128 v1 of n buffers (paper Sec. 5.1: a hash of the
 * transferred data stands in for the data; this library's hash is defined
 * in FP128 v1 below).
 *
 *   ptrs[i]   device array of n device pointers; buffer i starts there.
 *             Any byte alignment is accepted (16-byte aligned buffers take
 *             the fast path).  May be null when sizes[i] == 0.
 *   sizes[i]  device array of n byte counts.
 *   out128[i] device array of n results.
 *
 * n == 0 is a no-op.  A buffer of size 0 gets the empty-input fingerprint.
 * Buffers may overlap or alias.  The result does not depend on the buffer's
 * address, on the other buffers of the batch or on the launch schedule.
 * Returns ODP_ERR_INVALID_ARG for null arrays with n > 0 and ODP_ERR_OOM /
 * ODP_ERR_CUDA for allocation / launch failures.  A null ptrs[i] with
 * sizes[i] > 0 is detected on the device: out128[i] is set to {0, 0} and
 * ODP_ERR_INVALID_ARG is recorded in the device status word read by
 * odp_fingerprint_status.
 *
 * FP128 v1 (all arithmetic modulo 2^64; C[i] = output i of SplitMix64
 * seeded with 0x46503132385F7631, "FP128_v1"; Kodd(i) = C[i] | 1):
 *   - split the input into 4096-byte chunks; the last one holds r valid
 *     bytes and is zero-padded; a chunk is 256 little-endian 16-byte words
 *     (lo, hi);
 *   - lane l = 0..31 absorbs words l, l+32, ..., l+224 into two chains
 *     a = C[32+2l], b = C[33+2l]:  a = S(a ^ lo; Kodd 0, 1),
 *     b = S(b ^ hi; Kodd 2, 3) with S(v; k1, k2) = ((v*k1) ^ (v*k1) >> 32) * k2;
 *     then a ^= b * Kodd(4); b ^= a * Kodd(5);
 *   - the 32 lane states combine as a complete binary tree with
 *     node = L ^ G(R), G(x, y) = (y, x ^ y);
 *   - leaf = M_Q(root.x ^ r ^ C[18], root.y ^ C[19]);
 *   - leaves combine in a left-balanced binary tree (split at the largest
 *     power of two below the count) with node = M_P(L.x ^ G(R).x ^ count,
 *     L.y ^ G(R).y ^ C[20]), count = leaves under the node;
 *   - out = M_Z(root.x ^ len, root.y ^ nchunks ^ C[21]); the empty input
 *     uses root = (C[22], C[23]);
 *   - M_{Q,P,Z}(x, y) with four odd multipliers k0..k3 (Kodd 6-9, 10-13,
 *     14-17): x*=k0; y^=x>>29; y*=k1; x^=y>>32; x*=k2; y^=x>>32; y*=k3;
 *     x^=y>>29.
 */
int odp_fingerprint(const void* const* ptrs, const uint64_t* sizes, uint64_t n,
                    odp_fp128* out128, cudaStream_t stream);

/*
 * odp_fingerprint_noalloc -- the same results as odp_fingerprint, computed
 * without allocating any device memory.  The paper has no counterpart; this
 * is for callers that cannot call cudaMalloc or an allocator at the moment
 * they need a fingerprint (code running inside an allocator or an
 * out-of-memory path, or a host program that forbids allocation after
 * start-up).  Its scratch is one file-scope device array of about 0.9 MiB
 * that every GPU loading the library keeps until the process exits.
 *
 *   ptrs, sizes, out128: as for odp_fingerprint (device arrays, n entries).
 *   n: at most 4096 buffers; larger n returns ODP_ERR_UNSUPPORTED.  Buffers
 *   of any size are accepted (large batches use larger tiles).
 *
 * The first call on each device looks up the array's device address (with
 * that device current) and may return ODP_ERR_CUDA if that fails; make the
 * first call on a device before capturing a stream.  The address is kept
 * until the process exits: do not call this after cudaDeviceReset on a
 * device it has already been called on.  Every call reuses the same array:
 * calls whose work overlaps on the GPU (different streams, or another
 * thread) race and give wrong results, so serialise them.  Each call clears
 * the array's header and tree counters first, so a racing or failed call
 * spoils only its own results and those of the calls it overlapped.  A null
 * ptrs[i] with sizes[i] > 0 yields {0, 0} in out128[i]; this variant does
 * not update the status word of odp_fingerprint_status.
 */
int odp_fingerprint_noalloc(const void* const* ptrs, const uint64_t* sizes, uint64_t n,
                            odp_fp128* out128, cudaStream_t stream);

/*
 * Launch schedule of the fingerprint kernels.  A schedule spreads the work
 * differently over the GPU and never changes a fingerprint (tiles are
 * aligned power-of-two blocks of chunks; the left-balanced tree gives the
 * same root for any tile size).
 *   warps_per_cta  4, 8 or 16
 *   ctas_per_sm    0 = as many as fit, else at most this many
 *   tmin_scale     >= 1; each buffer aims at tmin_scale * (resident warps) / n
 *                  tiles of 1..32 chunks
 *   load_stages    0: chunks are read with 16-byte register loads; 2 or 4:
 *                  whole chunks of 16-byte-aligned buffers are bulk-copied
 *                  (cp.async.bulk) into that many shared-memory slots per
 *                  warp (not with 16 warps and 4 slots)
 */
typedef struct odp_fp_schedule {
    int32_t warps_per_cta;
    int32_t ctas_per_sm;
    int32_t tmin_scale;
    int32_t load_stages;
} odp_fp_schedule;

/*
 * odp_fingerprint_one -- FP128 of one device buffer given by a host-side
 * pointer and size (no device argument arrays to copy first); the launch is
 * sized to the buffer, which saves the idle warps of a full grid on small
 * buffers.  out128 is device memory (16 bytes).  Asynchronous like
 * odp_fingerprint; size 0 gives the empty-input hash; a null ptr with
 * size > 0 writes zero and records ODP_ERR_INVALID_ARG in the status word
 * (odp_fingerprint_status).  No paper counterpart: a host-side convenience
 * for tools that fingerprint one transfer at a time.
 */
int odp_fingerprint_one(const void* ptr, uint64_t size, odp_fp128* out128, cudaStream_t stream);

/* odp_fingerprint with an explicit schedule (ODP_ERR_INVALID_ARG for values
 * outside the ranges above). */
int odp_fingerprint_with(const odp_fp_schedule* sched, const void* const* ptrs,
                         const uint64_t* sizes, uint64_t n, odp_fp128* out128,
                         cudaStream_t stream);

/*
 * odp_autotune_fingerprint -- times every candidate schedule on this input
 * (`reps` timed calls each after one warm-up; synchronises `stream`), checks
 * that all candidates give identical fingerprints (ODP_ERR_MISMATCH if not),
 * and records the fastest for n's size class (bit length of n).  Later
 * odp_fingerprint calls of that class use it.  When the environment variable
 * ODP_AUTOTUNE_CACHE names a file, the table is read from it on first use and
 * rewritten after each tuning.  out128 ends with the fingerprints; *best and
 * *best_ms (optional) receive the choice and its time per call.
 */
int odp_autotune_fingerprint(const void* const* ptrs, const uint64_t* sizes, uint64_t n,
                             odp_fp128* out128, cudaStream_t stream, int reps,
                             odp_fp_schedule* best, float* best_ms);

/* Forgets every tuned schedule (in memory; the cache file is left alone). */
int odp_autotune_clear(void);

/* Reads (synchronising `stream`) and clears the device status word that
 * odp_fingerprint writes for per-buffer errors; *status receives ODP_OK or
 * the first error recorded. */
int odp_fingerprint_status(cudaStream_t stream, int32_t* status);

/* -------------------------------------------------------------- analysis */

/* Event kinds (OMPT target data-op types plus target kernel launches). */
enum {
    ODP_ALLOC = 1,
    ODP_TO_DEV = 2,      /* host -> device transfer */
    ODP_FROM_DEV = 3,    /* device -> host transfer */
    ODP_DEV_TO_DEV = 4,  /* device -> device transfer */
    ODP_DELETE = 5,
    ODP_KERNEL = 6
};

#define ODP_HOST_DEVICE (-1)
#define ODP_MAX_SITES 65536u
#define ODP_MAX_BYTES (1ull << 56)
#define ODP_NO_EVENT (~0ull)
/* odp_event.flags bit for odp_server_submit: fp_lo/fp_hi already hold the
 * transfer's fingerprint (taken when the bytes were known to be in place);
 * the server uses it and ignores the payload pointer. */
#define ODP_EVENT_FP_GIVEN 0x1u

/*
 * One mapping event, 64 bytes, packed little-endian (the paper's log entry
 * of Sec. 5: start/end time, hash of the transferred data, source and
 * destination device, code location, bytes, operation type; Sec. 7.4 sizes
 * it at 72 B -- this record replaces the code pointer by a site id).
 *   - t_start_ns / t_end_ns: interval of the operation (kernels too).
 *   - host_addr: host address of the mapped variable; dev_addr: device
 *     address (alloc/delete pairing key together with dst_dev).
 *   - fp_lo/fp_hi: FP128 of the transferred bytes (transfers only).
 *   - src_dev/dst_dev: device numbers, host = -1.  ALLOC, DELETE and KERNEL
 *     use dst_dev for their device.
 *   - site_id: caller-assigned code-location id (< ODP_MAX_SITES).
 *   - flags: ODP_EVENT_FP_GIVEN (serving only); odp_analyze ignores them.
 */
#pragma pack(push, 1)
typedef struct odp_event {
    uint64_t t_start_ns;
    uint64_t t_end_ns;
    uint64_t host_addr;
    uint64_t dev_addr;
    uint64_t bytes;
    uint64_t fp_lo;
    uint64_t fp_hi;
    uint32_t site_id;
    uint8_t kind;
    int8_t src_dev;
    int8_t dst_dev;
    uint8_t flags;
} odp_event;

/* Finding kinds (Sec. 7.5 abbreviations). */
enum { ODP_DD = 1, ODP_RT = 2, ODP_RA = 3, ODP_UA = 4, ODP_UT = 5 };

/*
 * One finding, 48 bytes.
 *   DD: event = a transfer whose <fingerprint, destination> was received
 *       before; partner = the first such transfer (Alg. 1).
 *   RT: event = a transfer tx, partner = the reception rx it pairs with
 *       (Alg. 2, literal peek/dequeue semantics); the wasted trip is rx.
 *   RA: event = the alloc of a repeated <host_addr, device, bytes> pair,
 *       partner = the first pair's alloc (Alg. 3).
 *   UA: event = an unused allocation, partner = its delete or ODP_NO_EVENT
 *       when it is never deleted (Alg. 4).
 *   UT: event = an unused to-device transfer; partner = the transfer that
 *       overwrote it, or ODP_NO_EVENT after the last kernel (Alg. 5).
 *   wasted_bytes / wasted_ns: bytes and duration of the eliminable
 *   operations (DD, UT: the event; RT: rx; RA, UA: alloc + delete).
 */
typedef struct odp_finding {
    uint8_t kind;
    uint8_t pad0[3];
    uint32_t site;          /* site_id of `event` */
    uint32_t partner_site;  /* site_id of `partner`, 0xFFFFFFFF if none */
    uint32_t pad1;
    uint64_t event;
    uint64_t partner;
    uint64_t wasted_bytes;
    uint64_t wasted_ns;
} odp_finding;

/* Per (kind, site) totals, rows ordered by (kind, site). */
typedef struct odp_site_row {
    uint32_t site;
    uint8_t kind;
    uint8_t pad[3];
    uint64_t count;
    uint64_t wasted_bytes;
    uint64_t wasted_ns;
} odp_site_row;

/* Trace totals and the Sec. 7.6 estimate: predicted time = span - saved,
 * where saved sums the durations of the union of wasted events; the
 * predicted speedup is speedup_num / speedup_den (den 0: unbounded). */
typedef struct odp_summary {
    uint64_t n_events, n_transfers, n_allocs, n_deletes, n_kernels;
    uint64_t n_pairs, n_unpaired_allocs, n_unmatched_deletes;
    uint64_t count[6];          /* indexed by finding kind */
    uint64_t wasted_bytes[6];
    uint64_t wasted_ns[6];
    uint64_t trace_begin_ns, trace_end_ns, trace_span_ns;
    uint64_t saved_ns;
    uint64_t speedup_num, speedup_den;
} odp_summary;
#pragma pack(pop)

/* Output description for odp_analyze.  All pointers are device pointers. */
typedef struct odp_findings {
    odp_finding* items;        /* capacity entries, 16-byte aligned */
    uint64_t capacity;
    uint64_t* count;           /* total findings (may exceed capacity) */
    odp_site_row* sites;       /* sites_capacity rows */
    uint64_t sites_capacity;
    uint64_t* sites_count;     /* total rows (may exceed sites_capacity) */
    odp_summary* summary;
    int32_t* status;           /* ODP_OK, ODP_WARN_TRUNCATED or an error */
} odp_findings;

/*
 * odp_analyze -- Algorithms 1-5 of Sec. 5 over n events (device memory,
 * 16-byte aligned, else ODP_ERR_INVALID_ARG; chronological: t_start_ns
 * nondecreasing, array index breaks ties).
 *
 * Findings are written ordered by (kind, event index).  If the total
 * exceeds out->capacity the first `capacity` are written, *count still holds
 * the total and *status is ODP_WARN_TRUNCATED; the summary and the site rows
 * are always computed over all findings.  Validation errors (unknown kind,
 * t_end < t_start, zero-byte transfer, inconsistent devices, site_id or
 * bytes beyond the limits -> ODP_ERR_MALFORMED; decreasing t_start ->
 * ODP_ERR_UNSORTED; the lowest offending index decides) zero the outputs and
 * set *status.  n must be below 2^32 - 16 (ODP_ERR_UNSUPPORTED otherwise).
 * Interpretations where the paper is silent: transfers only for Alg. 1/2,
 * to-device transfers only for Alg. 5, a DELETE closes the nearest earlier
 * open ALLOC of the same (device, dev_addr), never-deleted allocations end
 * at the trace end for Alg. 4 and are excluded from Alg. 3.
 */
int odp_analyze(const odp_event* events, uint64_t n, const odp_findings* out,
                cudaStream_t stream);

/* ---------------------------------------------------------------- serving */

/*
 * A serving loop (no counterpart in the paper, which analyses its log after
 * the program exits): many host threads submit mapping events as they
 * happen; the server merges them in start-time order behind a watermark,
 * forms batches continuously, fingerprints every transfer's payload on the
 * GPU, appends the events to a log resident in device memory and updates
 * state kept on the device for Algorithm 1 (duplicate transfers), Algorithm
 * 2 (round trips; in a content group that shows a third endpoint a round
 * trip can depend on receptions still to come, so the group's round trips
 * from then on are reported by odp_server_flush, which replays Alg. 2's
 * queues over the group), the alloc/delete pairing, Algorithm 3 (repeated
 * allocations), Algorithm 4 (unused allocations: a pair is decided once a kernel on its device
 * overlaps it or the merged stream has passed its delete's end) and
 * Algorithm 5 (unused transfers: decided when the next kernel of the
 * transfer's device arrives), so those findings are reported while the
 * program runs.  A completed pair whose <host address, device, bytes> key
 * still has an allocation open waits until none is (that allocation, once
 * completed, could be the key's first pair).  After odp_server_flush the
 * streamed findings equal odp_analyze's over the same log unless a capacity
 * overflowed (stream_overflow); odp_analyze over the resident log
 * (odp_server_log) is exact always.
 */
typedef struct odp_server odp_server;

typedef struct odp_server_cfg {
    int32_t device;                 /* CUDA device of the server */
    int32_t n_slots;                /* batches in flight at most (>= 1) */
    uint64_t device_budget_bytes;   /* device memory the server may use */
    uint64_t max_events;            /* capacity of the resident log */
    uint32_t max_batch_events;      /* events per batch at most */
    uint32_t max_producers;         /* distinct submitting threads at most */
    uint32_t watermark_timeout_us;  /* a thread silent this long stops holding
                                       back the merge watermark */
    uint32_t batch_interval_us;     /* batcher polling period */
} odp_server_cfg;

/* Per-server counters and latency percentiles (ns, from the submit call of
 * the event that completes a finding to the moment the server hands the
 * finding to the poll queue). */
typedef struct odp_server_stats {
    uint64_t events_submitted, events_processed, batches, findings_streamed;
    uint64_t late_events;           /* events behind the released watermark
                                       (they break the log's order) */
    uint64_t latency_p50_ns, latency_p99_ns, latency_max_ns;
    uint64_t first_submit_ns, last_done_ns;  /* steady-clock stamps */
    uint64_t rt_groups_at_flush;    /* content groups with > 2 endpoints: their
                                       round trips after the third endpoint
                                       appeared are reported at the flush */
    uint64_t stream_overflow;       /* findings, and decisions waiting for a
                                       later event, that did not fit the
                                       server's capacities (3 * max_batch_events
                                       + min(max_events, 16 * max_batch_events)
                                       + 64 findings per batch; that minimum of
                                       waiting pairs and transfers): the streamed
                                       findings then miss them; odp_analyze over
                                       the log stays exact */
    uint64_t queue_p50_ns, queue_p99_ns;  /* the part of the latency before the
                                       reporting batch was launched (merge
                                       watermark and batch formation) */
    uint64_t device_bytes;          /* device memory the server allocated
                                       (at most odp_server_bytes) */
} odp_server_stats;

/*
 * Device bytes a server with this configuration reserves (*bytes): every
 * block odp_server_create allocates, plus per slot the scratch of the slot's
 * fingerprint calls (their plan for max_batch_events buffers) and 20 MB for
 * allocation granularity.  Host arithmetic only (no device call).  ODP_ERR_INVALID_ARG for a null argument or a zero field
 * (n_slots < 1), ODP_ERR_UNSUPPORTED for max_events or max_batch_events above
 * 2^30.
 */
int odp_server_bytes(const odp_server_cfg* cfg, uint64_t* bytes);

/* Creates a server and allocates all of its device memory up front.  The
 * budget is checked first, before any device call: ODP_ERR_OOM if
 * odp_server_bytes exceeds a non-zero device_budget_bytes, or if the device
 * refuses an allocation.  Other errors as odp_server_bytes. */
int odp_server_create(const odp_server_cfg* cfg, odp_server** out);

/*
 * Registers the calling thread as a producer before its first event.  Until
 * the thread submits, the merge watermark does not pass start_t_ns, so its
 * first events cannot fall behind events already released from other
 * threads.  A thread that submits without attaching is registered by its
 * first submit (and may then see its first events counted as late).
 */
int odp_server_attach(odp_server* s, uint64_t start_t_ns);

/*
 * Opens an event on the calling thread (registering the thread if needed):
 * *t_start_ns receives its start time on the server's clock (steady clock,
 * ns), to be used as the event's t_start_ns.  A thread that has called begin
 * once announces its events: the merge watermark waits for it only while it
 * has events open (at the start of the earliest), and otherwise passes it at
 * the server's current time instead of waiting for its next submit.  Such a
 * thread must begin every event it submits.  Submitting an event closes the
 * latest open event that starts no later than it; odp_server_cancel closes
 * one without submitting it; an event open longer than watermark_timeout_us
 * stops holding the watermark.  Returns ODP_ERR_INVALID_ARG for a null
 * argument, ODP_ERR_UNSUPPORTED past the producer limit.
 */
int odp_server_begin(odp_server* s, uint64_t* t_start_ns);

/* Closes the calling thread's open event that started at t_start_ns without
 * submitting it (ODP_ERR_INVALID_ARG if no such event is open). */
int odp_server_cancel(odp_server* s, uint64_t t_start_ns);

/*
 * Thread-safe.  Submits n events (host memory, 64-byte records).  For
 * transfers, dev_payloads[i] is the device address of the transferred bytes
 * (event.bytes of them); the server computes fp_lo/fp_hi, unless the event's
 * flags carry ODP_EVENT_FP_GIVEN (then the record's fingerprint is used and
 * dev_payloads[i] is ignored; it may be null).  Events of one
 * calling thread must have nondecreasing t_start_ns.  Returns
 * ODP_ERR_INVALID_ARG for null arrays, ODP_ERR_UNSUPPORTED when the log
 * capacity or the producer limit would be exceeded.
 */
int odp_server_submit(odp_server* s, const odp_event* host_events,
                      const void* const* dev_payloads, uint64_t n);

/* Moves up to cap streamed findings (all five kinds; event indices in the
 * merged log order) to host_out; *n_out receives the number moved. */
int odp_server_poll(odp_server* s, odp_finding* host_out, uint64_t cap, uint64_t* n_out);

/* Releases every submitted event (the watermark no longer waits), blocks
 * until all batches are done, and ends the trace for Algorithms 4 and 5:
 * pairs still waiting for a kernel are unused, allocations never deleted are
 * unused unless a kernel seen on their device ends at or after their start,
 * and to-device transfers still waiting for a kernel come after the last one;
 * content groups with more than two endpoints get their round trips by a
 * replay of Alg. 2's queues over the group's transfers, reporting those not
 * streamed before (these findings carry no latency).  Events submitted after
 * a flush extend the log; findings already reported are not revisited. */
int odp_server_flush(odp_server* s);

/* The resident merged log (device pointer) and its length; valid until the
 * next submit or destroy.  Pass it to odp_analyze for Algorithms 1-5. */
int odp_server_log(odp_server* s, const odp_event** dev_log, uint64_t* n);

/* Maps merged-log positions to (submitting thread index, sequence number of
 * the event within that thread's submissions); host arrays of n entries. */
int odp_server_origin(odp_server* s, uint32_t* producer, uint64_t* seq, uint64_t n);

int odp_server_stats_get(odp_server* s, odp_server_stats* st);

int odp_server_destroy(odp_server* s);

/* ----------------------------------------------- fingerprints of a log */

/*
 * odp_fingerprint_log -- writes the FP128 v1 fingerprint of every transfer's
 * bytes into that transfer's record (fp_lo, fp_hi), all transfers of the log
 * in one batched odp_fingerprint call.  The paper (Sec. 5) stores a hash of
 * the transferred data in each data-op record; this is that step for a log
 * whose payloads are still in device memory, in the batched form instead of
 * one launch per transfer.
 *
 *   events    device, n 64-byte records, 8-byte aligned.  Records of kind
 *             ODP_TO_DEV, ODP_FROM_DEV or ODP_DEV_TO_DEV get their fp_lo and
 *             fp_hi overwritten with the fingerprint of `bytes` bytes at
 *             payloads[i]; every other record is left unchanged.
 *   payloads  device array of n device pointers (any alignment); entries of
 *             non-transfers are not read.  A null pointer with bytes > 0
 *             gives {0, 0} and records ODP_ERR_INVALID_ARG in the status
 *             word of odp_fingerprint_status.
 * Asynchronous on `stream`; scratch from the library's allocator (32 bytes
 * per record plus the fingerprint plan).  ODP_ERR_INVALID_ARG for null
 * arrays with n > 0 or a misaligned `events`.
 */
int odp_fingerprint_log(odp_event* events, const void* const* payloads, uint64_t n,
                        cudaStream_t stream);

/* ------------------------------------------------------- collision check */

/*
 * odp_verify_fingerprints -- the collision check of the paper's App. B:
 * where two transfers carry the same fingerprint, compare the transferred
 * bytes.  Every transfer of the log is compared with the first transfer
 * (lowest index) that has its fingerprint; a different length or any
 * different byte is a collision, i.e. a duplicate or round trip the
 * fingerprint would report falsely (the paper observed none).
 *
 *   events       device, n 64-byte records, 16-byte aligned
 *   payloads     device array of n device pointers: the bytes of each
 *                transfer (event.bytes of them, any alignment); entries of
 *                other events are ignored
 *   n_collisions device u64: number of colliding transfers
 *   flags        device, n bytes, or null: 1 for a colliding transfer, 0 for
 *                a verified one; other events' bytes are left unchanged
 * Asynchronous on `stream`; scratch from the library's allocator.
 */
int odp_verify_fingerprints(const odp_event* events, const void* const* payloads, uint64_t n,
                            unsigned long long* n_collisions, uint8_t* flags,
                            cudaStream_t stream);

/* ----------------------------------------------------------------- memory */

typedef void* (*odp_alloc_fn)(size_t bytes, cudaStream_t stream, void* ctx);
typedef void (*odp_free_fn)(void* ptr, cudaStream_t stream, void* ctx);

/* Installs the scratch allocator (null restores cudaMallocAsync/FreeAsync).
 * Frees every cached scratch block first (synchronising the device). */
int odp_set_allocator(odp_alloc_fn alloc_fn, odp_free_fn free_fn, void* ctx);

/* Releases all cached scratch memory and graphs (synchronises the device). */
int odp_release_scratch(void);

#ifdef __cplusplus
}
#endif

#endif /* ODP_H */
