// server.cu -- continuous-batching serving loop over mapping events.
//
// Producers (any host threads) submit events as they happen.  A batcher
// thread merges them in start-time order behind a watermark (the smallest,
// over producers that submitted recently, of the last start time; for a
// producer that opens its events with odp_server_begin, the start of its
// earliest open event, or the current time if none is open), cuts batches and
// runs each through a slot: the payloads of its transfers are fingerprinted
// on the slot's own stream (slots overlap), then, in order on the analysis
// stream, the batch is appended to the log resident in device memory and the
// state of Algorithms 1-5 kept in device tables is updated: by one block
// (srv_batch_small) for batches of up to 2,048 events, else by a CUDA graph
// of the same steps captured per slot.  Each producer has its own lock;
// findings are copied to pinned host memory and handed to the poll queue
// with their latency.
//
// Streaming Alg. 1: table <fingerprint> -> first log index (content id) and
// table <content id, destination> -> first receiver persist across batches;
// log indices grow with time, so the minimum is the first ever.
// Streaming Alg. 2 (content groups with at most two endpoints): a transfer
// from A pairs with the first later reception of its content at A.  Inside
// a batch that is the next run of destinations in the batch's content-sorted
// transfers; transfers left unpaired wait in a per-<content id, endpoint>
// list, which the first reception at that endpoint in a later batch closes.
// Groups that ever show a third endpoint stop streaming round trips: what a
// transfer pairs with may then depend on receptions still to come.  Every
// group's transfers are kept linked in log order, and odp_server_flush walks
// the groups with more than two endpoints with the literal queues of Alg. 2
// (per endpoint: receptions counted, a cursor at the front of its queue) and
// reports the round trips that were not streamed.  Those streamed while the
// group had two endpoints stay exact: a transfer from A to B follows every
// earlier reception at A, so they all succeed, and its partner is the first
// later reception at A, which comes before any event of a third endpoint.
// Streaming pairs and Alg. 3: a table <device address, device> holds the top
// of each address's stack of open allocations (links per log index); a
// DELETE closes the nearest open ALLOC, in batch order per address.  Per
// <host address, device, bytes> key, a second table counts the key's open
// allocations and keeps its first completed pair's alloc; each batch walks its
// allocations and completed pairs key by key in log order.  A completed pair
// waits in its key's list while another allocation of the key is open (that
// one, completed later, could be the key's first pair); when none is open,
// every waiting pair of the key is decided against the first, which no later
// allocation can precede.  The flush decides what still waits (allocations
// never deleted are not pairs).
// Streaming Alg. 4: an allocation is used iff some kernel on its device
// overlaps [alloc start, delete end].  Kernels of earlier batches are summed
// up by their largest end per device; the pair's batch's kernels are indexed
// per device (start order, running maximum of ends) and searched by
// bisection; a pair still undecided waits in a list until a batch starts
// after its delete ends (no later kernel can overlap it) or a kernel of a
// later batch overlaps it.  Flush ends the trace: waiting pairs are unused,
// and allocations never deleted are checked against every kernel seen.
// Streaming Alg. 5: a to-device transfer that starts while a kernel of its
// device runs (largest kernel end seen >= its start) is a barrier; any other
// waits for its device's next kernel, so the transfers of one device between
// two kernel arrivals form a segment (numbered by the kernels seen).  Per
// <host address, device> the latest waiting transfer is kept; a transfer that
// follows one of the same segment overwrites it, which is reported when the
// next kernel closes the segment (unless that kernel starts exactly when the
// later transfer does, which makes it a barrier).  Transfers still waiting at
// the flush come after the last kernel.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "common.cuh"
#include "fingerprint.cuh"
#include "prims.cuh"

namespace odp {
namespace {

using prim::Key128;
using prim::NONE32;
using prim::Table;

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr uint32_t EP_MORE = 1u << 16;  // endpoint set: more than two endpoints
constexpr int SRV_NDEV = 129;            // host + devices 0..127
constexpr uint64_t SRV_MAX_CAPACITY = 1ull << 30;  // max_events, max_batch_events

struct SrvDev {
    odp_event* log;
    uint32_t* cid;     // per log index (transfers)
    uint32_t* gtail;   // per content id: the group's last transfer so far (NONE32: none)
    uint32_t* glink;   // per log index: the next transfer of its content group (log order)
    uint8_t* rt_done;  // per log index: a round trip of this transfer has been reported
    uint32_t* next;    // per log index: pending-list links (transfers), open-alloc stack links
    Table t_fp, t_dd, t_pend, t_ep, t_b;
    Table t_pair;      // <device address, device> -> top of the open-alloc stack
    Table t_rid;       // <host address, device, bytes> -> first completed pair's alloc
    uint32_t* rid_open;  // per t_rid slot: open allocations of the key
    uint32_t* rid_wait;  // per t_rid slot: last waiting pair's alloc (NONE32: none)
    uint32_t* wait_next; // per log index (alloc of a waiting pair): the key's previous one
    uint32_t* wait_del;  // per log index (alloc of a waiting pair): its delete
    unsigned long long* kmax;  // per device: 1 + largest kernel end seen (0: none)
    uint2* pend[2];    // pairs waiting for the Alg. 4 decision (alloc, delete), ping-pong
    uint32_t* npend;   // [2] counts, [2] overflow count
    uint32_t pend_cap;
    Table t_ut;        // <host address, device> -> latest waiting to-device transfer
    uint32_t* kcnt;    // per device: kernels seen (the current segment number)
    uint32_t* useg;    // per log index: segment of a waiting to-device transfer
    uint2* utf[2];     // overwrites waiting for their segment to close (earlier, later), ping-pong
    uint32_t* utopen[2];  // to-device transfers still waiting for a kernel, ping-pong
    uint32_t* nut;     // [0..1] overwrite counts, [2..3] waiting counts, [4] overflow
    uint32_t* cur;     // which of the ping-pong lists is current (flipped per batch)
};

// Per-batch parameters, staged from the host with the batch, so that the
// analysis launch sequence is one CUDA graph replayed for every batch.
struct BatchPar {
    uint32_t nx;      // transfers in the batch
    uint32_t nf;      // of them, fingerprinted by the server
    uint32_t m;       // events in the batch
    uint32_t hlen;    // sort scratch: histogram length of the current pass
    uint64_t g0;      // log index of the batch's first event
    uint64_t t_next;  // largest start released so far: every later event starts at or after it
};

struct SlotDev {
    odp_event* ev;         // batch events (staged from host)
    const void** ptrs;     // payload pointers of the batch's transfers
    uint64_t* sizes;
    odp_fp128* fp;
    uint32_t* xpos;        // batch position of each transfer
    uint32_t* fpos;        // batch position of each transfer the server fingerprints
    BatchPar* par;         // the batch's parameters (device copy)
    uint32_t* nx;          // = &par->nx: [0] transfers, [1] of them fingerprinted here
    uint32_t* sfp;         // per batch position: slot in t_fp / t_dd / t_b
    uint32_t* sdd;
    uint32_t* sb;
    uint32_t* skeys;       // content-sorted transfers (key, value) + alternates
    uint32_t* svals;
    prim::SortTmp sort;
    odp_finding* find;     // streamed findings of the batch
    uint64_t* complete;    // log index of the event that completed each finding
    uint32_t* nfind;
    uint32_t* pa;          // pairs completed in the batch: alloc, delete
    uint32_t* pd;
    uint32_t* dalloc;      // per batch position of a DELETE: the alloc it closed (NONE32: none)
    uint32_t* rslot;       // their slot in t_rid
    uint32_t* bk;          // kernels of the batch (log indices), by device, in log order
    uint32_t* bktmp;       // the same in log order
    unsigned long long* end1;  // per bk entry: 1 + largest end among its device's kernels up to it
    uint32_t* kst;         // [256] per device: first bk entry
    uint32_t* kcn;         // [256] per device: number of bk entries
    uint32_t* cnt;         // [0] pairs, [1] kernels, [2] overwrites, [3] waiting transfers
};

// The batch's kernels on `dev`: how many come before log index g and the
// largest end among those (0: none), the total on dev, and the first one
// after g (NONE32: none).
struct BatchKernels {
    uint32_t before, total, first_after;
    unsigned long long max_end1;  // 1 + largest end of those before g
};

__device__ __forceinline__ BatchKernels batch_kernels_on(const SlotDev& s, uint32_t dev,
                                                         uint32_t g) {
    const uint32_t st = s.kst[dev], c = s.kcn[dev];
    uint32_t lo = 0, hi = c;  // first entry of the device's run with log index >= g
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s.bk[st + mid] < g) lo = mid + 1;
        else hi = mid;
    }
    BatchKernels r;
    r.before = lo;
    r.total = c;
    r.first_after = lo < c ? s.bk[st + lo] : NONE32;
    r.max_end1 = lo ? s.end1[st + lo - 1] : 0ull;
    return r;
}

__device__ __forceinline__ uint32_t ep_of(int8_t dev) { return (uint32_t)(dev + 1) & 0xFF; }

__device__ __forceinline__ bool is_xfer(uint8_t k) {
    return k == ODP_TO_DEV || k == ODP_FROM_DEV || k == ODP_DEV_TO_DEV;
}

__device__ __forceinline__ void emit(const SlotDev& s, uint32_t cap, const odp_event* log,
                                     uint8_t kind, uint64_t e, uint64_t p, uint64_t wasted_of,
                                     uint64_t completing) {
    const uint32_t j = atomicAdd(s.nfind, 1u);
    if (j >= cap) return;
    store_finding(s.find, j, kind, log[e].site_id, log[p].site_id, e, p, log[wasted_of].bytes,
                  log[wasted_of].t_end_ns - log[wasted_of].t_start_ns);
    s.complete[j] = completing;
}

__device__ __forceinline__ uint64_t dur_of(const odp_event& e) { return e.t_end_ns - e.t_start_ns; }

// A round trip <tx e, rx p> (the wasted trip is p), marked as reported.
__device__ __forceinline__ void emit_rt(const SrvDev& d, const SlotDev& s, uint32_t cap, uint64_t e,
                                        uint64_t p, uint64_t completing) {
    d.rt_done[e] = 1;
    emit(s, cap, d.log, ODP_RT, e, p, p, completing);
}

// A finding with explicit wasted bytes and time; partner NONE32 = none.
__device__ __forceinline__ void emit_w(const SlotDev& s, uint32_t cap, const odp_event* log,
                                       uint8_t kind, uint64_t e, uint32_t p, uint64_t wb,
                                       uint64_t wn, uint64_t completing) {
    const uint32_t j = atomicAdd(s.nfind, 1u);
    if (j >= cap) return;
    const bool np = p == NONE32;
    store_finding(s.find, j, kind, log[e].site_id, np ? 0xFFFFFFFFu : log[p].site_id, e,
                  np ? ODP_NO_EVENT : (uint64_t)p, wb, wn);
    s.complete[j] = completing;
}

// Fingerprints into the batch's transfer records.
__global__ void srv_scatter_fp(SlotDev s) {
    const uint32_t nf = s.nx[1];
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += gridDim.x * blockDim.x) {
        odp_event& e = s.ev[s.fpos[j]];
        e.fp_lo = s.fp[j].lo;
        e.fp_hi = s.fp[j].hi;
    }
}

// Content ids: insert <fingerprint> with the log index.
__device__ __forceinline__ void srv_insert_fp_body(SrvDev d, SlotDev s) {
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m, cap = *d.t_fp.cap_dev;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
        const odp_event& e = d.log[g0 + q];
        s.sfp[q] = is_xfer(e.kind) ? prim::table_insert_min(d.t_fp, cap, Key128{e.fp_lo, e.fp_hi},
                                                            (uint32_t)(g0 + q))
                                   : NONE32;
    }
}

__global__ void srv_insert_fp(SrvDev d, SlotDev s) { srv_insert_fp_body(d, s); }

// cid; first-receiver and batch-first-receiver tables; endpoint sets.
__device__ __forceinline__ void srv_insert_dd_body(SrvDev d, SlotDev s) {
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m;
    const uint32_t cap_dd = *d.t_dd.cap_dev, cap_b = *d.t_b.cap_dev, cap_ep = *d.t_ep.cap_dev;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
        const uint64_t g = g0 + q;
        const odp_event& e = d.log[g];
        if (!is_xfer(e.kind) || s.sfp[q] == NONE32) {
            s.sdd[q] = s.sb[q] = NONE32;
            continue;
        }
        const uint32_t cid = d.t_fp.slots[s.sfp[q]].v;
        d.cid[g] = cid;
        const Key128 k{(uint64_t)cid | ((uint64_t)ep_of(e.dst_dev) << 32), 0};
        s.sdd[q] = prim::table_insert_min(d.t_dd, cap_dd, k, (uint32_t)g);
        s.sb[q] = prim::table_insert_min(d.t_b, cap_b, k, (uint32_t)g);
        // endpoint set of the content group: up to two endpoints, then "more"
        const uint32_t es = prim::table_insert_min(d.t_ep, cap_ep, Key128{cid, 1}, NONE32);
        if (es == NONE32) continue;
        for (uint32_t ep : {ep_of(e.src_dev), ep_of(e.dst_dev)}) {
            uint32_t cur = d.t_ep.slots[es].v;
            for (int it = 0; it < 64; ++it) {  // bounded CAS loop
                uint32_t a = cur == NONE32 ? 0 : cur;
                const uint32_t e1 = a & 0xFF, e2 = (a >> 8) & 0xFF;
                const uint32_t v = ep + 1;
                uint32_t nxt;
                if (a & EP_MORE || e1 == v || e2 == v) break;
                if (e1 == 0) nxt = a | v;
                else if (e2 == 0) nxt = a | (v << 8);
                else nxt = a | EP_MORE;
                const uint32_t old = atomicCAS(&d.t_ep.slots[es].v, cur, nxt);
                if (old == cur) break;
                cur = old;
            }
        }
    }
}

__global__ void srv_insert_dd(SrvDev d, SlotDev s) { srv_insert_dd_body(d, s); }

__device__ __forceinline__ bool complex_group(const SrvDev& d, uint32_t cid) {
    const uint32_t cap = *d.t_ep.cap_dev;
    const uint32_t es = prim::table_insert_min(d.t_ep, cap, Key128{cid, 1}, NONE32);
    const uint32_t v = es == NONE32 ? EP_MORE : d.t_ep.slots[es].v;
    return v != NONE32 && (v & EP_MORE);
}

// Duplicate transfers, and the first reception of each group at each
// endpoint in this batch closes the round trips waiting for it.
__device__ __forceinline__ void srv_dd_resolve_body(SrvDev d, SlotDev s, uint32_t cap,
                                                    uint64_t max_events) {
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m, cap_pend = *d.t_pend.cap_dev;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
        if (s.sdd[q] == NONE32) continue;
        const uint64_t g = g0 + q;
        const uint32_t first = d.t_dd.slots[s.sdd[q]].v;
        if (first != (uint32_t)g) emit(s, cap, d.log, ODP_DD, g, first, g, g);
        if (d.t_b.slots[s.sb[q]].v != (uint32_t)g) continue;  // not the batch's first here
        const uint32_t cid = d.cid[g];
        if (complex_group(d, cid)) continue;
        const Key128 k{(uint64_t)cid | ((uint64_t)ep_of(d.log[g].dst_dev) << 32), 2};
        const uint32_t ps = prim::table_insert_min(d.t_pend, cap_pend, k, NONE32);
        if (ps == NONE32) continue;
        uint32_t e = atomicExch(&d.t_pend.slots[ps].v, NONE32);
        for (uint64_t guard = 0; e != NONE32 && guard < max_events; ++guard) {
            emit_rt(d, s, cap, e, g, g);
            e = d.next[e];
        }
    }
}

__global__ void srv_dd_resolve(SrvDev d, SlotDev s, uint32_t cap, uint64_t max_events) {
    srv_dd_resolve_body(d, s, cap, max_events);
}

// Sort keys: content id of each transfer, value = batch position.
__device__ __forceinline__ void srv_sort_keys_body(SrvDev d, SlotDev s) {
    const uint64_t g0 = s.par->g0;
    const uint32_t nx = *s.nx;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nx; j += gridDim.x * blockDim.x) {
        const uint32_t q = s.xpos[j];
        s.skeys[j] = d.cid[g0 + q];
        s.svals[j] = q;
    }
}

__global__ void srv_sort_keys(SrvDev d, SlotDev s) { srv_sort_keys_body(d, s); }

// In-batch round trips on the content-sorted transfers: the partner of a
// transfer is the first event of the next destination run of its group;
// transfers without one wait in the group's list for their source.
__device__ __forceinline__ void srv_rt_batch_body(SrvDev d, SlotDev s, uint32_t cap) {
    const uint64_t g0 = s.par->g0;
    const uint32_t nx = *s.nx;
    const uint32_t cap_pend = *d.t_pend.cap_dev;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nx; r += gridDim.x * blockDim.x) {
        const uint32_t cid = s.skeys[r];
        if (complex_group(d, cid)) continue;
        const uint64_t g = g0 + s.svals[r];
        const uint32_t dst = ep_of(d.log[g].dst_dev);
        uint32_t t = r + 1;
        while (t < nx && s.skeys[t] == cid && ep_of(d.log[g0 + s.svals[t]].dst_dev) == dst) ++t;
        if (t < nx && s.skeys[t] == cid) {
            const uint64_t p = g0 + s.svals[t];
            emit_rt(d, s, cap, g, p, p);
        } else {
            const Key128 k{(uint64_t)cid | ((uint64_t)ep_of(d.log[g].src_dev) << 32), 2};
            const uint32_t ps = prim::table_insert_min(d.t_pend, cap_pend, k, NONE32);
            if (ps == NONE32) continue;
            const uint32_t old = atomicExch(&d.t_pend.slots[ps].v, (uint32_t)g);
            d.next[g] = old;
        }
    }
}

__global__ void srv_rt_batch(SrvDev d, SlotDev s, uint32_t cap) { srv_rt_batch_body(d, s, cap); }

// Appends the batch's transfers to their content groups' lists, in log order:
// in the content-sorted transfers (stable, so log order inside a group) each
// run links its members, and the run's head links the group's previous tail.
__device__ __forceinline__ void srv_group_link_body(SrvDev d, SlotDev s) {
    const uint64_t g0 = s.par->g0;
    const uint32_t nx = *s.nx;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nx; r += gridDim.x * blockDim.x) {
        const uint32_t cid = s.skeys[r];
        const uint32_t g = (uint32_t)(g0 + s.svals[r]);
        const bool more = r + 1 < nx && s.skeys[r + 1] == cid;
        d.glink[g] = more ? (uint32_t)(g0 + s.svals[r + 1]) : NONE32;
        if (r > 0 && s.skeys[r - 1] == cid) continue;
        uint32_t t = r;
        while (t + 1 < nx && s.skeys[t + 1] == cid) ++t;
        const uint32_t old = d.gtail[cid];
        if (old != NONE32) d.glink[old] = g;
        d.gtail[cid] = (uint32_t)(g0 + s.svals[t]);
    }
}

__global__ void srv_group_link(SrvDev d, SlotDev s) { srv_group_link_body(d, s); }

// Alloc/delete events of the batch keyed by their <device address, device>
// slot (other events sort last); value = batch position.
__device__ __forceinline__ void srv_pair_keys_body(SrvDev d, SlotDev s) {
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m;
    const uint32_t cap = *d.t_pair.cap_dev, none_key = d.t_pair.cap_max + 1;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
        const odp_event& e = d.log[g0 + q];
        uint32_t k = none_key;
        if (e.kind == ODP_ALLOC || e.kind == ODP_DELETE) {
            const uint32_t sl = prim::table_insert(d.t_pair, cap, Key128{e.dev_addr, ep_of(e.dst_dev)});
            if (sl != NONE32) k = sl;
        }
        s.skeys[q] = k;
        s.svals[q] = q;
    }
}

__global__ void srv_pair_keys(SrvDev d, SlotDev s) { srv_pair_keys_body(d, s); }

// One thread per address group of the batch (sorted, batch order inside)
// walks it: ALLOC pushes on the address's open-alloc stack, DELETE pops the
// nearest open ALLOC and records the pair.  Kernels of the batch are listed.
__device__ __forceinline__ void srv_pair_walk_body(SrvDev d, SlotDev s) {
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m;
    const uint32_t none_key = d.t_pair.cap_max + 1;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        const uint32_t k = s.skeys[r];
        if (k == none_key || (r > 0 && s.skeys[r - 1] == k)) continue;
        uint32_t top = d.t_pair.slots[k].v;
        for (uint32_t t = r; t < m && s.skeys[t] == k; ++t) {
            const uint32_t g = (uint32_t)(g0 + s.svals[t]);
            if (d.log[g].kind == ODP_ALLOC) {
                d.next[g] = top;
                top = g;
            } else if (top != NONE32) {
                const uint32_t i = atomicAdd(&s.cnt[0], 1u);
                s.pa[i] = top;
                s.pd[i] = g;
                s.dalloc[s.svals[t]] = top;
                top = d.next[top];
            } else {
                s.dalloc[s.svals[t]] = NONE32;  // no open allocation: unmatched
            }
        }
        d.t_pair.slots[k].v = top;
    }
}

__global__ void srv_pair_walk(SrvDev d, SlotDev s) { srv_pair_walk_body(d, s); }

__device__ __forceinline__ Key128 rid_key(const odp_event& e) {
    return Key128{e.host_addr, e.bytes | ((uint64_t)ep_of(e.dst_dev) << 56)};
}

// Alg. 3 sort keys: the batch's allocations by their own <host address,
// device, bytes> slot, and its completed pairs (at their delete) by their
// alloc's slot; other events sort last.  Value = batch position.
__device__ __forceinline__ void srv_ra_keys_body(SrvDev d, SlotDev s) {
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m;
    const uint32_t cap = *d.t_rid.cap_dev, none_key = d.t_rid.cap_max + 1;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
        const odp_event& e = d.log[g0 + q];
        uint32_t k = none_key;
        if (e.kind == ODP_ALLOC) {
            k = prim::table_insert(d.t_rid, cap, rid_key(e));
        } else if (e.kind == ODP_DELETE && s.dalloc[q] != NONE32) {
            k = prim::table_insert(d.t_rid, cap, rid_key(d.log[s.dalloc[q]]));
        }
        s.skeys[q] = k == NONE32 ? none_key : k;
        s.svals[q] = q;
    }
}

__global__ void srv_ra_keys(SrvDev d, SlotDev s) { srv_ra_keys_body(d, s); }

__device__ __forceinline__ void ra_decide(const SrvDev& d, const SlotDev& s, uint32_t cap,
                                          uint32_t a, uint32_t first, uint64_t completing) {
    if (a == first) return;
    const odp_event& ea = d.log[a];
    const uint32_t del = d.wait_del[a];
    emit_w(s, cap, d.log, ODP_RA, a, first, ea.bytes, dur_of(ea) + dur_of(d.log[del]), completing);
}

// One thread per key of the batch walks its allocations and completions in
// log order (see the header comment).
__device__ __forceinline__ void srv_ra_walk_body(SrvDev d, SlotDev s, uint32_t cap,
                                                 uint64_t max_events) {
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m;
    const uint32_t none_key = d.t_rid.cap_max + 1;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        const uint32_t k = s.skeys[r];
        if (k == none_key || (r > 0 && s.skeys[r - 1] == k)) continue;
        uint32_t open = d.rid_open[k], first = d.t_rid.slots[k].v, wait = d.rid_wait[k];
        for (uint32_t t = r; t < m && s.skeys[t] == k; ++t) {
            const uint32_t q = s.svals[t];
            const uint32_t g = (uint32_t)(g0 + q);
            if (d.log[g].kind == ODP_ALLOC) {
                ++open;
                continue;
            }
            const uint32_t a = s.dalloc[q];  // a completed pair (a, g)
            if (open > 0) --open;
            first = min(first, a);
            d.wait_del[a] = g;
            d.wait_next[a] = wait;
            wait = a;
            if (open == 0) {  // no allocation of the key is open: decide the waiting pairs
                uint64_t guard = 0;
                for (uint32_t x = wait; x != NONE32 && guard < max_events; x = d.wait_next[x], ++guard)
                    ra_decide(d, s, cap, x, first, g);
                wait = NONE32;
            }
        }
        d.rid_open[k] = open;
        d.t_rid.slots[k].v = first;
        d.rid_wait[k] = wait;
    }
}

__global__ void srv_ra_walk(SrvDev d, SlotDev s, uint32_t cap, uint64_t max_events) {
    srv_ra_walk_body(d, s, cap, max_events);
}

// Some kernel of the batch on `dev` overlaps [lo, hi]: of the device's
// kernels that start by hi (a prefix: the log is in start order), the
// latest end reaches lo.
__device__ __forceinline__ bool batch_kernel_overlaps(const SrvDev& d, const SlotDev& s,
                                                      uint32_t dev, uint64_t lo, uint64_t hi) {
    const uint32_t st = s.kst[dev], c = s.kcn[dev];
    uint32_t a = 0, b = c;  // kernels with t_start <= hi
    while (a < b) {
        const uint32_t mid = (a + b) >> 1;
        if (d.log[s.bk[st + mid]].t_start_ns <= hi) a = mid + 1;
        else b = mid;
    }
    return a > 0 && s.end1[st + a - 1] > lo;
}

// Alg. 4 for the batch's pairs (against earlier kernels, then the batch's)
// and for the waiting pairs (against the batch's kernels); undecided pairs
// whose delete ends before t_next (the start of every later event) are
// unused, the rest wait in list `nxt`.
__device__ __forceinline__ void srv_ua_body(SrvDev d, SlotDev s, uint32_t cap) {
    const uint64_t t_next = s.par->t_next;
    const uint32_t cur = *d.cur, nxt = cur ^ 1;
    const uint32_t n_new = s.cnt[0], n_old = min(d.npend[cur], d.pend_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_new + n_old;
         i += gridDim.x * blockDim.x) {
        const bool fresh = i < n_new;
        const uint32_t a = fresh ? s.pa[i] : d.pend[cur][i - n_new].x;
        const uint32_t g = fresh ? s.pd[i] : d.pend[cur][i - n_new].y;
        const odp_event& ea = d.log[a];
        const odp_event& eg = d.log[g];
        const uint32_t dev = ep_of(ea.dst_dev);
        bool used = false;
        if (fresh) {
            const unsigned long long km = d.kmax[dev];
            used = km != 0 && km - 1 >= ea.t_start_ns;
        }
        if (!used) used = batch_kernel_overlaps(d, s, dev, ea.t_start_ns, eg.t_end_ns);
        if (used) continue;
        if (eg.t_end_ns < t_next) {
            emit_w(s, cap, d.log, ODP_UA, a, g, ea.bytes, dur_of(ea) + dur_of(eg), g);
        } else {
            const uint32_t j = atomicAdd(&d.npend[nxt], 1u);
            if (j < d.pend_cap) d.pend[nxt][j] = make_uint2(a, g);
            else atomicAdd(&d.npend[2], 1u);
        }
    }
}

__global__ void srv_ua(SrvDev d, SlotDev s, uint32_t cap) { srv_ua_body(d, s, cap); }

// Also flips the current waiting lists: the last kernel of a batch to read them.
__device__ __forceinline__ void srv_kmax_body(SrvDev d, SlotDev s) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *d.cur ^= 1u;
    const uint32_t nk = s.cnt[1];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += gridDim.x * blockDim.x) {
        const odp_event& k = d.log[s.bk[i]];
        atomicMax(&d.kmax[ep_of(k.dst_dev)], (unsigned long long)k.t_end_ns + 1ull);
        atomicAdd(&d.kcnt[ep_of(k.dst_dev)], 1u);
    }
}

__global__ void srv_kmax(SrvDev d, SlotDev s) { srv_kmax_body(d, s); }

// To-device transfers of the batch: barriers drop out; a waiting transfer
// gets its segment and is keyed by its <host address, device> slot (others
// sort last).
__device__ __forceinline__ void srv_ut_keys_body(SrvDev d, SlotDev s) {
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m;
    const uint32_t cap = *d.t_ut.cap_dev, none_key = d.t_ut.cap_max + 1;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
        const uint32_t g = (uint32_t)(g0 + q);
        const odp_event& e = d.log[g];
        uint32_t k = none_key;
        if (e.kind == ODP_TO_DEV) {
            const uint32_t dev = ep_of(e.dst_dev);
            const BatchKernels bk = batch_kernels_on(s, dev, g);
            const unsigned long long km = max(d.kmax[dev], bk.max_end1);
            if (!(km != 0 && km - 1 >= e.t_start_ns)) {
                d.useg[g] = d.kcnt[dev] + bk.before;
                const uint32_t sl = prim::table_insert(d.t_ut, cap, Key128{e.host_addr, dev});
                if (sl != NONE32) k = sl;
            }
        }
        s.skeys[q] = k;
        s.svals[q] = q;
    }
}

__global__ void srv_ut_keys(SrvDev d, SlotDev s) { srv_ut_keys_body(d, s); }

// One thread per <host address, device> group of the batch, in order: a
// transfer that follows the key's latest waiting transfer in the same
// segment records an overwrite (into s.pa/s.pd, count s.cnt[2]); every
// waiting transfer is listed (s.rslot, count s.cnt[3]).
__device__ __forceinline__ void srv_ut_walk_body(SrvDev d, SlotDev s) {
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m;
    const uint32_t none_key = d.t_ut.cap_max + 1;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        const uint32_t k = s.skeys[r];
        if (k == none_key || (r > 0 && s.skeys[r - 1] == k)) continue;
        uint32_t last = d.t_ut.slots[k].v;
        for (uint32_t t = r; t < m && s.skeys[t] == k; ++t) {
            const uint32_t g = (uint32_t)(g0 + s.svals[t]);
            if (last != NONE32 && d.useg[last] == d.useg[g]) {
                const uint32_t j = atomicAdd(&s.cnt[2], 1u);
                s.pa[j] = last;
                s.pd[j] = g;
            }
            s.rslot[atomicAdd(&s.cnt[3], 1u)] = g;
            last = g;
        }
        d.t_ut.slots[k].v = last;
    }
}

__global__ void srv_ut_walk(SrvDev d, SlotDev s) { srv_ut_walk_body(d, s); }

// Overwrites and waiting transfers, carried from earlier batches (list cur)
// and new in this one: an overwrite whose segment a kernel of this batch
// closes is reported if the later transfer starts before that kernel (else
// it is a barrier); transfers whose segment stays open carry over to list
// cur ^ 1.
__device__ __forceinline__ void srv_ut_resolve_body(SrvDev d, SlotDev s, uint32_t cap) {
    const uint32_t cur = *d.cur, nxt = cur ^ 1;
    const uint32_t n_f = min(d.nut[cur], d.pend_cap), n_fb = s.cnt[2];
    const uint32_t n_o = min(d.nut[2 + cur], d.pend_cap), n_ob = s.cnt[3];
    const uint32_t n_all = n_f + n_fb + n_o + n_ob;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_all; i += gridDim.x * blockDim.x) {
        if (i < n_f + n_fb) {
            const uint32_t c = i < n_f ? d.utf[cur][i].x : s.pa[i - n_f];
            const uint32_t t = i < n_f ? d.utf[cur][i].y : s.pd[i - n_f];
            const uint32_t dev = ep_of(d.log[t].dst_dev);
            const BatchKernels bk = batch_kernels_on(s, dev, t);
            if (bk.first_after == NONE32) {  // segment still open
                const uint32_t j = atomicAdd(&d.nut[nxt], 1u);
                if (j < d.pend_cap) d.utf[nxt][j] = make_uint2(c, t);
                else atomicAdd(&d.nut[4], 1u);
            } else if (d.log[t].t_start_ns < d.log[bk.first_after].t_start_ns) {
                emit_w(s, cap, d.log, ODP_UT, c, t, d.log[c].bytes, dur_of(d.log[c]),
                       bk.first_after);
            }
        } else {
            const uint32_t o = i - n_f - n_fb;
            const uint32_t g = o < n_o ? d.utopen[cur][o] : s.rslot[o - n_o];
            const uint32_t dev = ep_of(d.log[g].dst_dev);
            if (batch_kernels_on(s, dev, g).first_after == NONE32) {
                const uint32_t j = atomicAdd(&d.nut[2 + nxt], 1u);
                if (j < d.pend_cap) d.utopen[nxt][j] = g;
                else atomicAdd(&d.nut[4], 1u);
            }
        }
    }
}

__global__ void srv_ut_resolve(SrvDev d, SlotDev s, uint32_t cap) {
    srv_ut_resolve_body(d, s, cap);
}

// Flush: every waiting pair is unused (no kernel follows the end of the
// trace); every allocation still open is checked against all kernels seen,
// with the end of the trace as its delete end; every to-device transfer still
// waiting for a kernel comes after the last one.
__global__ void srv_flush(SrvDev d, SlotDev s, uint32_t cap, uint64_t max_events) {
    const uint32_t cur = *d.cur;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t n_old = min(d.npend[cur], d.pend_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_old; i += stride) {
        const uint32_t a = d.pend[cur][i].x, g = d.pend[cur][i].y;
        emit_w(s, cap, d.log, ODP_UA, a, g, d.log[a].bytes, dur_of(d.log[a]) + dur_of(d.log[g]),
               ~0ull);
    }
    const uint32_t n_open = min(d.nut[2 + cur], d.pend_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_open; i += stride) {
        const uint32_t g = d.utopen[cur][i];
        emit_w(s, cap, d.log, ODP_UT, g, NONE32, d.log[g].bytes, dur_of(d.log[g]), ~0ull);
    }
    // Alg. 3: pairs still waiting for an allocation of their key that was
    // never deleted (not a pair) are decided against the key's first pair
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= d.t_rid.cap_max; k += stride) {
        const uint32_t w = d.rid_wait[k];
        if (w == NONE32) continue;
        const uint32_t first = d.t_rid.slots[k].v;
        uint64_t guard = 0;
        for (uint32_t x = w; x != NONE32 && guard < max_events; x = d.wait_next[x], ++guard)
            ra_decide(d, s, cap, x, first, ~0ull);
        d.rid_wait[k] = NONE32;
    }
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= d.t_pair.cap_max; k += stride) {
        uint32_t a = d.t_pair.slots[k].v;
        for (uint64_t guard = 0; a != NONE32 && guard < max_events; ++guard) {
            const odp_event& ea = d.log[a];
            const unsigned long long km = d.kmax[ep_of(ea.dst_dev)];
            if (!(km != 0 && km - 1 >= ea.t_start_ns))
                emit_w(s, cap, d.log, ODP_UA, a, NONE32, ea.bytes, dur_of(ea), ~0ull);
            a = d.next[a];
        }
    }
}

// Flush, Alg. 2 for the content groups with more than two endpoints: one
// thread per group replays the literal queues over the group's list: a
// transfer from A peeks at the front of A's queue (the receptions at A, all
// of the group's, in order) and, if there is one, reports the round trip and
// pops the front of its destination's queue.  Round trips already reported
// (streamed before the third endpoint, or by an earlier round or flush) are
// skipped; a round trip is marked reported only when it fit the findings
// buffer, so the host repeats the replay until a round drops nothing.
__global__ void srv_mx_flush(SrvDev d, SlotDev s, uint32_t cap, uint64_t n_log,
                             uint64_t max_events) {
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < n_log;
         g += (uint64_t)gridDim.x * blockDim.x) {
        if (!is_xfer(d.log[g].kind) || d.cid[g] != (uint32_t)g) continue;  // not a group's first
        if (!complex_group(d, (uint32_t)g)) continue;
        uint32_t nrx[SRV_NDEV], popped[SRV_NDEV], front[SRV_NDEV];
        for (int k = 0; k < SRV_NDEV; ++k) nrx[k] = popped[k] = 0, front[k] = NONE32;
        uint64_t guard = 0;
        for (uint32_t x = (uint32_t)g; x != NONE32 && guard < max_events; x = d.glink[x], ++guard) {
            const uint32_t b = ep_of(d.log[x].dst_dev);
            if (nrx[b]++ == 0) front[b] = x;
        }
        guard = 0;
        for (uint32_t x = (uint32_t)g; x != NONE32 && guard < max_events; x = d.glink[x], ++guard) {
            const uint32_t a = ep_of(d.log[x].src_dev), b = ep_of(d.log[x].dst_dev);
            if (popped[a] >= nrx[a]) continue;  // A's queue is empty: no round trip
            if (!d.rt_done[x]) {
                const uint32_t j = atomicAdd(s.nfind, 1u);
                if (j < cap) {
                    const uint32_t p = front[a];
                    store_finding(s.find, j, ODP_RT, d.log[x].site_id, d.log[p].site_id, x, p,
                                  d.log[p].bytes, dur_of(d.log[p]));
                    s.complete[j] = ~0ull;
                    d.rt_done[x] = 1;
                }
            }
            if (++popped[b] < nrx[b]) {  // pop B's front: move to its next reception
                uint32_t y = d.glink[front[b]];
                for (uint64_t k = 0; y != NONE32 && ep_of(d.log[y].dst_dev) != b && k < max_events;
                     ++k)
                    y = d.glink[y];
                front[b] = y;
            }
        }
    }
}

__global__ void srv_zero(uint32_t* p) { *p = 0; }

// First step of a batch: append its events to the log; reset the batch's
// counters and the counts of the next waiting lists.
__device__ __forceinline__ void srv_append_body(SrvDev d, SlotDev s) {
    const uint32_t m = s.par->m;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *s.nfind = 0;
        s.cnt[0] = s.cnt[1] = s.cnt[2] = s.cnt[3] = 0;
        const uint32_t nxt = *d.cur ^ 1u;
        d.npend[nxt] = 0;
        d.nut[nxt] = 0;
        d.nut[2 + nxt] = 0;
    }
    const uint4* src = reinterpret_cast<const uint4*>(s.ev);
    uint4* dst = reinterpret_cast<uint4*>(d.log + s.par->g0);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * m; i += gridDim.x * blockDim.x)
        dst[i] = src[i];
}

__global__ void srv_append(SrvDev d, SlotDev s) { srv_append_body(d, s); }

// The batch's kernels grouped by device, in log (= start) order within each
// device, with the running maximum of their ends (one block; three ordered
// passes: compaction, stable scatter by device, per-device max scan).  The
// questions Alg. 4 and 5 ask about the batch's kernels then become binary
// searches; s.cnt[1] receives the count.
constexpr int BKI_THREADS = 1024;

// wdev_sm: W x 256 words of shared memory for the per-warp device counts.
__device__ __forceinline__ void srv_bk_index_body(SrvDev d, SlotDev s, uint32_t* wdev_sm) {
    constexpr int W = BKI_THREADS / 32;
    __shared__ uint32_t wofs[W + 1];
    __shared__ uint32_t dbase[256];
    uint32_t(*wdev)[256] = reinterpret_cast<uint32_t(*)[256]>(wdev_sm);
    const uint64_t g0 = s.par->g0;
    const uint32_t m = s.par->m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1;
    for (int i = threadIdx.x; i < 256; i += BKI_THREADS) dbase[i] = 0;
    // 1. compaction of the batch's kernels in log order; counts per device
    uint32_t nk = 0;
    for (uint32_t c0 = 0; c0 < m; c0 += BKI_THREADS) {
        const uint32_t q = c0 + threadIdx.x;
        const bool isk = q < m && d.log[g0 + q].kind == ODP_KERNEL;
        const uint32_t bal = __ballot_sync(ODP_FULL_MASK, isk);
        if (lane == 0) wofs[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            const uint32_t v = wofs[lane];
            uint32_t incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(ODP_FULL_MASK, incl, o);
                if (lane >= o) incl += t;
            }
            wofs[lane] = incl - v;
            if (lane == 31) wofs[W] = incl;
        }
        __syncthreads();
        if (isk) {
            s.bktmp[nk + wofs[warp] + __popc(bal & lt)] = (uint32_t)(g0 + q);
            atomicAdd(&dbase[ep_of(d.log[g0 + q].dst_dev)], 1u);
        }
        nk += wofs[W];
        __syncthreads();
    }
    // 2. device runs: exclusive scan of the 256 counts (thread t owns device t)
    if (threadIdx.x < 256) {
        const uint32_t c = dbase[threadIdx.x];
        s.kcn[threadIdx.x] = c;
        wdev[0][threadIdx.x] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < 256; ++t) {
            const uint32_t c = wdev[0][t];
            dbase[t] = run;
            s.kst[t] = run;
            run += c;
        }
        s.cnt[1] = nk;
    }
    __syncthreads();
    // 3. stable scatter by device, chunk by chunk in log order
    for (uint32_t c0 = 0; c0 < nk; c0 += BKI_THREADS) {
        const uint32_t i = c0 + threadIdx.x;
        const bool valid = i < nk;
        const uint32_t k = valid ? s.bktmp[i] : 0u;
        const uint32_t dev = valid ? ep_of(d.log[k].dst_dev) : 256u;
        for (int t = lane; t < 256; t += 32) wdev[warp][t] = 0;
        __syncwarp();
        const uint32_t peers = __match_any_sync(ODP_FULL_MASK, dev);
        if (valid && lane == __ffs(peers) - 1) wdev[warp][dev] = __popc(peers);
        __syncthreads();
        uint32_t tot = 0;
        if (threadIdx.x < 256) {
            for (int w = 0; w < W; ++w) {
                const uint32_t c = wdev[w][threadIdx.x];
                wdev[w][threadIdx.x] = tot;
                tot += c;
            }
        }
        __syncthreads();
        if (valid) s.bk[dbase[dev] + wdev[warp][dev] + __popc(peers & lt)] = k;
        __syncthreads();
        if (threadIdx.x < 256) dbase[threadIdx.x] += tot;
        __syncthreads();
    }
    // 4. running maximum of end + 1 along each device's run (warp per device)
    for (uint32_t dev = warp; dev < 256; dev += W) {
        const uint32_t st = s.kst[dev], c = s.kcn[dev];
        unsigned long long carry = 0;
        for (uint32_t j0 = 0; j0 < c; j0 += 32) {
            const uint32_t j = j0 + lane;
            unsigned long long v = j < c ? d.log[s.bk[st + j]].t_end_ns + 1ull : 0ull;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long t = __shfl_up_sync(ODP_FULL_MASK, v, o);
                if (lane >= o) v = max(v, t);
            }
            v = max(v, carry);
            if (j < c) s.end1[st + j] = v;
            carry = __shfl_sync(ODP_FULL_MASK, v, 31);
        }
    }
}

__global__ void __launch_bounds__(BKI_THREADS) srv_bk_index(SrvDev d, SlotDev s) {
    __shared__ uint32_t wdev[BKI_THREADS / 32 * 256];
    srv_bk_index_body(d, s, wdev);
}

// A batch of at most SRV_SMALL_BATCH events runs as one block: the steps of
// the batch graph (enqueue_analysis) in the same order, with block barriers
// instead of kernel boundaries (every step loops over the batch with all the
// threads it is given) and the three sorts in shared memory (sized for
// SRV_SMALL_BATCH items, so the block fits beside fingerprint blocks on an
// SM).  A small batch then costs one launch and no inter-kernel gaps.
constexpr uint32_t SRV_SMALL_BATCH = 2048;
constexpr int SRV_SMALL_THREADS = 1024;  // = BKI_THREADS = SMALL_SORT_THREADS

__global__ void __launch_bounds__(SRV_SMALL_THREADS)
srv_batch_small(SrvDev d, SlotDev s, uint32_t B, uint32_t cap, uint64_t max_events, int bits_cid,
                int bits_pair, int bits_ut, int bits_rid) {
    const uint32_t* m_dev = &s.par->m;
    srv_append_body(d, s);
    __syncthreads();
    extern __shared__ __align__(16) uint32_t small_sm[];  // the sorts' buffers, free until then
    srv_bk_index_body(d, s, small_sm);
    __syncthreads();
    prim::table_clear_body(d.t_b, m_dev, B);
    __syncthreads();
    srv_insert_fp_body(d, s);
    __syncthreads();
    srv_insert_dd_body(d, s);
    __syncthreads();
    srv_dd_resolve_body(d, s, cap, max_events);
    __syncthreads();
    srv_sort_keys_body(d, s);
    __syncthreads();
    prim::sort_small_body<SRV_SMALL_BATCH>(s.skeys, s.svals, s.nx, SRV_SMALL_BATCH, bits_cid);
    __syncthreads();
    srv_rt_batch_body(d, s, cap);
    __syncthreads();
    srv_group_link_body(d, s);
    __syncthreads();
    srv_pair_keys_body(d, s);
    __syncthreads();
    prim::sort_small_body<SRV_SMALL_BATCH>(s.skeys, s.svals, m_dev, SRV_SMALL_BATCH, bits_pair);
    __syncthreads();
    srv_pair_walk_body(d, s);
    __syncthreads();
    srv_ra_keys_body(d, s);
    __syncthreads();
    prim::sort_small_body<SRV_SMALL_BATCH>(s.skeys, s.svals, m_dev, SRV_SMALL_BATCH, bits_rid);
    __syncthreads();
    srv_ra_walk_body(d, s, cap, max_events);
    __syncthreads();
    srv_ua_body(d, s, cap);
    __syncthreads();
    srv_ut_keys_body(d, s);
    __syncthreads();
    prim::sort_small_body<SRV_SMALL_BATCH>(s.skeys, s.svals, m_dev, SRV_SMALL_BATCH, bits_ut);
    __syncthreads();
    srv_ut_walk_body(d, s);
    __syncthreads();
    srv_ut_resolve_body(d, s, cap);
    __syncthreads();
    srv_kmax_body(d, s);
}

// After the flush: the current waiting lists are empty.
__global__ void srv_flush_reset(SrvDev d) {
    const uint32_t cur = *d.cur;
    d.npend[cur] = 0;
    d.nut[cur] = 0;
    d.nut[2 + cur] = 0;
}

struct Pending {
    odp_event ev;
    const void* payload;
    uint64_t submit_ns;
    uint64_t seq;
};

// One submitting thread.  Its own mutex guards its state, so threads do not
// contend with each other; the batcher takes each producer's lock briefly.
struct Producer {
    std::mutex mu;
    std::deque<Pending> q;
    uint64_t last_t = 0;
    uint64_t last_seen = 0;
    uint64_t seq = 0;
    // Threads that open their events with odp_server_begin hold the merge
    // back only while events are open (at the earliest open start time).
    bool announces = false;
    std::multiset<uint64_t> open;  // start times of events begun, not yet submitted
};

struct Slot {
    SlotDev d;
    odp_event* h_ev = nullptr;
    const void** h_ptrs = nullptr;
    uint64_t* h_sizes = nullptr;
    uint32_t* h_xpos = nullptr;
    uint32_t* h_fpos = nullptr;
    BatchPar* h_par = nullptr;
    odp_finding* h_find = nullptr;
    uint64_t* h_complete = nullptr;
    uint32_t* h_nfind = nullptr;
    uint32_t eager = 0;  // findings copied back with the batch
    cudaStream_t fp_stream = nullptr;
    cudaEvent_t fp_done = nullptr, an_done = nullptr;
    cudaGraphExec_t an_graph = nullptr;  // the batch analysis (enqueue_analysis)
    bool busy = false;
    uint64_t g0 = 0;
    uint32_t m = 0;
    uint64_t t_launch = 0;  // when the batch was formed and launched
};

}  // namespace
}  // namespace odp

struct odp_server {
    odp_server_cfg cfg;
    std::mutex mu;
    uint64_t serial = 0;                        // unique per server (thread-local caches)
    std::map<uint64_t, uint32_t> producer_of;  // thread serial -> producer (mu)
    std::unique_ptr<odp::Producer[]> producers;  // max_producers of them
    std::atomic<uint32_t> n_producers{0};
    std::vector<std::deque<odp::Pending>> staged;  // batcher: released, not yet merged
    std::thread batcher;
    std::atomic<bool> stop{false};
    std::atomic<bool> flushing{false};
    std::condition_variable cv_done;
    std::atomic<uint64_t> submitted{0};
    std::atomic<uint64_t> first_submit{0};
    std::atomic<uint64_t> late{0};  // events behind the released watermark
    uint64_t released_t = 0;        // batcher thread
    // device
    odp::SrvDev d;
    std::vector<void*> dev_blocks;
    uint64_t dev_bytes = 0;  // sum of the dev_blocks' sizes
    cudaStream_t an_stream = nullptr;
    std::vector<odp::Slot> slots;
    uint32_t find_cap = 0;
    // merged events not yet in a batch (batcher thread)
    std::deque<odp::Pending> ready;
    std::deque<uint32_t> ready_prod;
    // host bookkeeping (guarded by mu)
    uint64_t n_log = 0;       // events released into the log
    uint64_t n_done = 0;      // events whose batch completed
    std::vector<uint64_t> submit_ns;
    std::vector<uint32_t> origin_prod;
    std::vector<uint64_t> origin_seq;
    std::deque<odp_finding> outq;
    std::vector<uint64_t> latencies;
    std::vector<uint64_t> queue_lat;  // submit -> launch of the reporting batch
    uint64_t batches = 0, streamed = 0, last_done = 0;
    uint64_t find_overflow = 0;  // findings past a batch's (or the flush's) capacity
    std::mutex an_mu;             // orders work enqueued on the analysis stream
    uint64_t t_released_max = 0;  // largest start time launched so far (batcher thread)
    odp::SlotDev fl;              // flush-time finding buffers (find, complete, nfind)
    odp_finding* h_fl_find = nullptr;
    uint32_t* h_fl_n = nullptr;
    std::atomic<int> error{ODP_OK};
    bool small_ok = false;  // srv_batch_small may take its shared memory
};

namespace odp {
namespace {

uint32_t pow2_at_least(uint64_t v) {
    uint64_t c = 1024;
    while (c < v) c <<= 1;
    return (uint32_t)c;
}

int alloc_dev(odp_server* s, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return ODP_ERR_OOM;
    }
    s->dev_blocks.push_back(*p);
    s->dev_bytes += bytes;
    return ODP_OK;
}

int make_table(odp_server* s, Table& t, uint32_t cap, uint32_t* cap_dev, cudaStream_t st) {
    t.cap_max = cap;
    t.cap_dev = cap_dev;
    int rc = alloc_dev(s, (void**)&t.slots, sizeof(prim::Slot) * ((size_t)cap + 1));
    if (rc) return rc;
    prim::table_clear<<<256, 256, 0, st>>>(t, nullptr, cap / 2);
    return ODP_OK;
}

// The analysis of one batch on stream `as`, in batch order: Alg. 1 and 2,
// pairs, Alg. 3 and 4, Alg. 5.  Captured once per slot into a CUDA graph;
// every value that changes between batches is read from the slot's
// parameter block, so one graph launch replays the whole sequence.
void enqueue_analysis(odp_server* S, Slot& sl, cudaStream_t as) {
    const uint32_t B = S->cfg.max_batch_events;
    const int grid = (int)std::min<uint32_t>(1024, (B + 255) / 256);
    const uint32_t* m_dev = &sl.d.par->m;
    srv_append<<<grid, 256, 0, as>>>(S->d, sl.d);
    srv_bk_index<<<1, BKI_THREADS, 0, as>>>(S->d, sl.d);
    prim::table_clear<<<64, 256, 0, as>>>(S->d.t_b, m_dev, B);
    srv_insert_fp<<<grid, 256, 0, as>>>(S->d, sl.d);
    srv_insert_dd<<<grid, 256, 0, as>>>(S->d, sl.d);
    srv_dd_resolve<<<grid, 256, 0, as>>>(S->d, sl.d, S->find_cap, S->cfg.max_events);
    srv_sort_keys<<<grid, 256, 0, as>>>(S->d, sl.d);
    prim::radix_sort(sl.d.skeys, sl.d.svals, sl.d.nx, B, prim::bit_length(S->cfg.max_events),
                     sl.d.sort, as);
    srv_rt_batch<<<grid, 256, 0, as>>>(S->d, sl.d, S->find_cap);
    srv_group_link<<<grid, 256, 0, as>>>(S->d, sl.d);
    srv_pair_keys<<<grid, 256, 0, as>>>(S->d, sl.d);
    prim::radix_sort(sl.d.skeys, sl.d.svals, m_dev, B, prim::bit_length(S->d.t_pair.cap_max + 1),
                     sl.d.sort, as);
    srv_pair_walk<<<grid, 256, 0, as>>>(S->d, sl.d);
    srv_ra_keys<<<grid, 256, 0, as>>>(S->d, sl.d);
    prim::radix_sort(sl.d.skeys, sl.d.svals, m_dev, B, prim::bit_length(S->d.t_rid.cap_max + 1),
                     sl.d.sort, as);
    srv_ra_walk<<<grid, 256, 0, as>>>(S->d, sl.d, S->find_cap, S->cfg.max_events);
    srv_ua<<<grid, 256, 0, as>>>(S->d, sl.d, S->find_cap);
    srv_ut_keys<<<grid, 256, 0, as>>>(S->d, sl.d);
    prim::radix_sort(sl.d.skeys, sl.d.svals, m_dev, B, prim::bit_length(S->d.t_ut.cap_max + 1),
                     sl.d.sort, as);
    srv_ut_walk<<<grid, 256, 0, as>>>(S->d, sl.d);
    srv_ut_resolve<<<grid, 256, 0, as>>>(S->d, sl.d, S->find_cap);
    srv_kmax<<<grid, 256, 0, as>>>(S->d, sl.d);
}

int capture_analysis(odp_server* S, Slot& sl) {
    prim::sort_small_ready();  // sets a kernel attribute: outside the capture
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return ODP_ERR_CUDA;
    int rc = ODP_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        rc = ODP_ERR_CUDA;
    } else {
        enqueue_analysis(S, sl, cs);
        if (cudaStreamEndCapture(cs, &g) != cudaSuccess ||
            cudaGraphInstantiate(&sl.an_graph, g, 0) != cudaSuccess)
            rc = ODP_ERR_CUDA;
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc) cudaGetLastError();
    return rc;
}

// Runs, on every slot, a fingerprint of small buffers and an empty batch
// through both analysis paths, so the first real batch does not pay for
// loading these kernels (modules are loaded on first use).  Empty batches
// append nothing and change no table; the waiting-list parity is reset.
int warm_up(odp_server* S) {
    const uint32_t B = S->cfg.max_batch_events;
    cudaStream_t as = S->an_stream;
    for (auto& sl : S->slots) {
        cudaStream_t fs = sl.fp_stream;
        const uint32_t nw = B >= 2 ? 2 : 1;  // two buffers take the planned path
        for (uint32_t j = 0; j < nw; ++j) {
            sl.h_ptrs[j] = reinterpret_cast<const uint8_t*>(sl.d.ev) + 16 * j;  // staged bytes
            sl.h_sizes[j] = 16;
        }
        *sl.h_par = BatchPar{0, 0, 0, 0, 0, 0};
        cudaMemcpyAsync(sl.d.ptrs, sl.h_ptrs, sizeof(void*) * nw, cudaMemcpyHostToDevice, fs);
        cudaMemcpyAsync(sl.d.sizes, sl.h_sizes, 8ull * nw, cudaMemcpyHostToDevice, fs);
        cudaMemcpyAsync(sl.d.par, sl.h_par, sizeof(BatchPar), cudaMemcpyHostToDevice, fs);
        if (fp_run((const void* const*)sl.d.ptrs, sl.d.sizes, nw, sl.d.fp, fs,
                   fp_schedule_for(nw)) != ODP_OK)
            return ODP_ERR_CUDA;
        cudaEventRecord(sl.fp_done, fs);
        cudaStreamWaitEvent(as, sl.fp_done, 0);
        if (S->small_ok)
            srv_batch_small<<<1, SRV_SMALL_THREADS, prim::small_sort_smem(SRV_SMALL_BATCH), as>>>(
                S->d, sl.d, B, S->find_cap, S->cfg.max_events, prim::bit_length(S->cfg.max_events),
                prim::bit_length(S->d.t_pair.cap_max + 1), prim::bit_length(S->d.t_ut.cap_max + 1),
                prim::bit_length(S->d.t_rid.cap_max + 1));
        if (cudaGraphLaunch(sl.an_graph, as) != cudaSuccess) return ODP_ERR_CUDA;
        if (cudaStreamSynchronize(fs) != cudaSuccess) return ODP_ERR_CUDA;
    }
    cudaMemsetAsync(S->d.cur, 0, 4, as);
    if (cudaStreamSynchronize(as) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return ODP_ERR_CUDA;
    return ODP_OK;
}

void launch_batch(odp_server* S, Slot& sl) {
    const uint32_t m = sl.m;
    cudaStream_t fs = sl.fp_stream, as = S->an_stream;
    uint32_t nx = 0, nf = 0;  // transfers; those whose payload the server fingerprints
    uint64_t t_next = S->t_released_max;
    for (uint32_t q = 0; q < m; ++q) {
        t_next = std::max(t_next, sl.h_ev[q].t_start_ns);
        const uint8_t k = sl.h_ev[q].kind;
        if (k != ODP_TO_DEV && k != ODP_FROM_DEV && k != ODP_DEV_TO_DEV) continue;
        sl.h_xpos[nx++] = q;
        if (!(sl.h_ev[q].flags & ODP_EVENT_FP_GIVEN)) {
            sl.h_sizes[nf] = sl.h_ev[q].bytes;
            sl.h_fpos[nf++] = q;
        }
    }
    S->t_released_max = t_next;
    *sl.h_par = BatchPar{nx, nf, m, 0, sl.g0, t_next};
    cudaMemcpyAsync(sl.d.ev, sl.h_ev, sizeof(odp_event) * m, cudaMemcpyHostToDevice, fs);
    cudaMemcpyAsync(sl.d.ptrs, sl.h_ptrs, sizeof(void*) * nf, cudaMemcpyHostToDevice, fs);
    cudaMemcpyAsync(sl.d.sizes, sl.h_sizes, 8ull * nf, cudaMemcpyHostToDevice, fs);
    cudaMemcpyAsync(sl.d.xpos, sl.h_xpos, 4ull * nx, cudaMemcpyHostToDevice, fs);
    cudaMemcpyAsync(sl.d.fpos, sl.h_fpos, 4ull * nf, cudaMemcpyHostToDevice, fs);
    cudaMemcpyAsync(sl.d.par, sl.h_par, sizeof(BatchPar), cudaMemcpyHostToDevice, fs);
    if (nf) {
        FpLaunch L = fp_schedule_for(nf);
        if (fp_run((const void* const*)sl.d.ptrs, sl.d.sizes, nf, sl.d.fp, fs, L) != ODP_OK)
            S->error = ODP_ERR_CUDA;
        srv_scatter_fp<<<64, 256, 0, fs>>>(sl.d);
    }
    cudaEventRecord(sl.fp_done, fs);

    // analysis, in batch order on one stream
    std::lock_guard<std::mutex> an_lk(S->an_mu);
    cudaStreamWaitEvent(as, sl.fp_done, 0);
    if (m <= SRV_SMALL_BATCH && S->small_ok) {
        const uint32_t B = S->cfg.max_batch_events;
        srv_batch_small<<<1, SRV_SMALL_THREADS, prim::small_sort_smem(SRV_SMALL_BATCH), as>>>(
            S->d, sl.d, B, S->find_cap, S->cfg.max_events, prim::bit_length(S->cfg.max_events),
            prim::bit_length(S->d.t_pair.cap_max + 1), prim::bit_length(S->d.t_ut.cap_max + 1),
            prim::bit_length(S->d.t_rid.cap_max + 1));
    } else if (cudaGraphLaunch(sl.an_graph, as) != cudaSuccess) {
        S->error = ODP_ERR_CUDA;
    }
    // copy back the count and the findings a batch of m events usually has
    // at most; harvest fetches the rest when there are more
    sl.eager = (uint32_t)std::min<uint64_t>(S->find_cap, 2ull * m + 256);
    cudaMemcpyAsync(sl.h_nfind, sl.d.nfind, 4, cudaMemcpyDeviceToHost, as);
    cudaMemcpyAsync(sl.h_find, sl.d.find, sizeof(odp_finding) * sl.eager, cudaMemcpyDeviceToHost, as);
    cudaMemcpyAsync(sl.h_complete, sl.d.complete, 8ull * sl.eager, cudaMemcpyDeviceToHost, as);
    cudaEventRecord(sl.an_done, as);
    if (cudaGetLastError() != cudaSuccess) S->error = ODP_ERR_CUDA;
}

// Moves releasable events into the ready queue in merged order (batcher
// thread).  The watermark is the smallest bound any producer puts on its
// future events; each bound is read under that producer's lock.  `now` is
// read before any of those locks, so an announcing producer with nothing
// open begins its next event (under its lock) at or after it.
void release(odp_server* S) {
    const uint64_t now = now_ns();
    const bool all = S->flushing.load();
    const uint64_t timeout = (uint64_t)S->cfg.watermark_timeout_us * 1000ull;
    const uint32_t np = S->n_producers.load(std::memory_order_acquire);
    uint64_t wm = ~0ull;
    if (!all) {
        for (uint32_t i = 0; i < np; ++i) {
            Producer& p = S->producers[i];
            std::lock_guard<std::mutex> lk(p.mu);
            if (now > p.last_seen + timeout && p.q.empty()) continue;  // silent producer
            if (!p.announces) {
                wm = std::min(wm, p.last_t);
                continue;
            }
            // an event open longer than the timeout was abandoned
            while (!p.open.empty() && *p.open.begin() + timeout < now) p.open.erase(p.open.begin());
            wm = std::min(wm, p.open.empty() ? now : *p.open.begin());
        }
    }
    // take the queue prefixes with t_start <= wm, then merge them
    bool any = false;
    for (uint32_t i = 0; i < np; ++i) {
        Producer& p = S->producers[i];
        std::lock_guard<std::mutex> lk(p.mu);
        while (!p.q.empty() && p.q.front().ev.t_start_ns <= wm) {
            S->staged[i].push_back(p.q.front());
            p.q.pop_front();
            any = true;
        }
    }
    while (any) {
        int best = -1;
        uint64_t bt = 0;
        for (uint32_t i = 0; i < np; ++i) {
            const auto& q = S->staged[i];
            if (q.empty()) continue;
            if (best < 0 || q.front().ev.t_start_ns < bt) {
                best = (int)i;
                bt = q.front().ev.t_start_ns;
            }
        }
        if (best < 0) break;
        const Pending& p = S->staged[best].front();
        if (p.ev.t_start_ns < S->released_t) S->late.fetch_add(1, std::memory_order_relaxed);
        S->released_t = std::max(S->released_t, p.ev.t_start_ns);
        S->ready.push_back(p);
        S->ready_prod.push_back((uint32_t)best);
        S->staged[best].pop_front();
    }
}

void harvest(odp_server* S, Slot& sl) {
    const uint32_t n = std::min(*sl.h_nfind, S->find_cap);
    if (n > sl.eager) {  // the slot's streams are idle until it is released
        const uint32_t e = sl.eager;
        cudaMemcpyAsync(sl.h_find + e, sl.d.find + e, sizeof(odp_finding) * (n - e),
                        cudaMemcpyDeviceToHost, sl.fp_stream);
        cudaMemcpyAsync(sl.h_complete + e, sl.d.complete + e, 8ull * (n - e),
                        cudaMemcpyDeviceToHost, sl.fp_stream);
        if (cudaStreamSynchronize(sl.fp_stream) != cudaSuccess) S->error = ODP_ERR_CUDA;
    }
    const uint64_t t = now_ns();
    std::lock_guard<std::mutex> lk(S->mu);
    S->find_overflow += *sl.h_nfind - n;
    for (uint32_t j = 0; j < n; ++j) {
        S->outq.push_back(sl.h_find[j]);
        const uint64_t c = sl.h_complete[j];
        if (c < S->submit_ns.size()) {
            const uint64_t t0 = S->submit_ns[c];
            S->latencies.push_back(t - t0);
            S->queue_lat.push_back(sl.t_launch > t0 ? sl.t_launch - t0 : 0);
        }
    }
    S->streamed += n;
    S->n_done += sl.m;
    S->last_done = t;
    ++S->batches;
    sl.busy = false;
    S->cv_done.notify_all();
}

void batcher_main(odp_server* S) {
    cudaSetDevice(S->cfg.device);
    const uint32_t B = S->cfg.max_batch_events;
    while (true) {
        bool idle = true;
        for (auto& sl : S->slots) {
            if (sl.busy && cudaEventQuery(sl.an_done) == cudaSuccess) {
                harvest(S, sl);
                idle = false;
            }
        }
        release(S);
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (auto& sl : S->slots) {
                if (S->ready.empty()) break;
                if (sl.busy) continue;
                const uint32_t m = (uint32_t)std::min<size_t>(B, S->ready.size());
                sl.g0 = S->n_log;
                sl.m = m;
                uint32_t nx = 0;
                for (uint32_t q = 0; q < m; ++q) {
                    const Pending& p = S->ready.front();
                    sl.h_ev[q] = p.ev;
                    const uint8_t k = p.ev.kind;
                    if ((k == ODP_TO_DEV || k == ODP_FROM_DEV || k == ODP_DEV_TO_DEV) &&
                        !(p.ev.flags & ODP_EVENT_FP_GIVEN))
                        sl.h_ptrs[nx++] = p.payload;
                    S->submit_ns[S->n_log] = p.submit_ns;
                    S->origin_prod[S->n_log] = S->ready_prod.front();
                    S->origin_seq[S->n_log] = p.seq;
                    ++S->n_log;
                    S->ready.pop_front();
                    S->ready_prod.pop_front();
                }
                sl.busy = true;
                sl.t_launch = now_ns();
                lk.unlock();
                launch_batch(S, sl);
                lk.lock();
                idle = false;
            }
            if (S->stop.load() && S->ready.empty()) {
                bool any = false;
                for (auto& sl : S->slots) any |= sl.busy;
                bool queued = false;
                const uint32_t np = S->n_producers.load(std::memory_order_acquire);
                for (uint32_t i = 0; i < np; ++i) {
                    std::lock_guard<std::mutex> plk(S->producers[i].mu);
                    queued |= !S->producers[i].q.empty();
                }
                if (!any && !queued) break;
            }
        }
        if (idle) std::this_thread::sleep_for(std::chrono::microseconds(S->cfg.batch_interval_us));
    }
}

}  // namespace
}  // namespace odp

extern "C" {

int odp_server_bytes(const odp_server_cfg* cfg, uint64_t* bytes) {
    using namespace odp;
    if (!cfg || !bytes) return ODP_ERR_INVALID_ARG;
    if (cfg->n_slots < 1 || cfg->max_events == 0 || cfg->max_batch_events == 0 ||
        cfg->max_producers == 0)
        return ODP_ERR_INVALID_ARG;
    // tables of 2 * capacity slots, rounded up to a power of two, index in 32 bits
    if (cfg->max_events > SRV_MAX_CAPACITY || cfg->max_batch_events > SRV_MAX_CAPACITY)
        return ODP_ERR_UNSUPPORTED;
    const uint64_t E = cfg->max_events, B = cfg->max_batch_events;
    const uint64_t cap_p = pow2_at_least(2 * E), cap_b = pow2_at_least(2 * B);
    const uint64_t pend_cap = std::min<uint64_t>(E, 16 * B);
    const uint64_t find_cap = 3 * B + pend_cap + 64;
    const uint64_t table = sizeof(prim::Slot);
    // the blocks odp_server_create allocates, plus per slot the scratch of the
    // slot's fingerprint calls and 20 MB for allocation granularity
    const uint64_t shared = 64 + E * (64 + 4 + 4 + 4 + 4 + 4 + 1 + 4 + 4) + 7 * table * (cap_p + 1) +
                            8 * (cap_p + 1) +
                            table * (cap_b + 1) + 12 * SRV_NDEV + 40 * pend_cap + 80 +
                            find_cap * (sizeof(odp_finding) + 8);
    const uint64_t hist = 4 * prim::sort_hist_words((uint32_t)B);
    const uint64_t scan = 4 * (prim::scan_tmp_words(256u * ((uint32_t)B / prim::SORT_TILE + 2)) + 16);
    const uint64_t per_slot = B * (sizeof(odp_event) + 8 + 8 + 16 + 4 + 4 + 13 * 4 + 8) +
                              sizeof(BatchPar) + hist + scan + find_cap * (sizeof(odp_finding) + 8) +
                              16 + 2 * 4 * 256 + 16 + fp_plan_scratch_bytes(B) + (20ull << 20);
    *bytes = shared + (uint64_t)cfg->n_slots * per_slot;
    return ODP_OK;
}

int odp_server_create(const odp_server_cfg* cfg, odp_server** out) {
    using namespace odp;
    if (!cfg || !out) return ODP_ERR_INVALID_ARG;
    uint64_t need = 0;
    int brc = odp_server_bytes(cfg, &need);
    if (brc != ODP_OK) return brc;
    // refused before any device call when the reservation exceeds the budget
    if (cfg->device_budget_bytes && need > cfg->device_budget_bytes) return ODP_ERR_OOM;
    if (cudaSetDevice(cfg->device) != cudaSuccess) return ODP_ERR_CUDA;
    const uint64_t E = cfg->max_events, B = cfg->max_batch_events;
    const uint32_t cap_p = pow2_at_least(2 * E), cap_b = pow2_at_least(2 * B);
    const uint32_t pend_cap = (uint32_t)std::min<uint64_t>(E, 16 * B);
    const uint64_t find_cap = 3 * B + pend_cap + 64;

    static std::atomic<uint64_t> next_server{1};
    odp_server* S = new odp_server();
    S->cfg = *cfg;
    S->serial = next_server.fetch_add(1);
    S->producers.reset(new odp::Producer[cfg->max_producers]);
    S->staged.resize(cfg->max_producers);
    S->find_cap = (uint32_t)find_cap;
    auto fail = [&](int rc) {
        odp_server_destroy(S);
        return rc;
    };
    if (cudaStreamCreateWithFlags(&S->an_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ODP_ERR_CUDA);
    uint32_t* caps = nullptr;
    int rc = alloc_dev(S, (void**)&caps, 64);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.log, sizeof(odp_event) * E);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.cid, 4 * E);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.next, 4 * E);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.gtail, 4 * E);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.glink, 4 * E);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.rt_done, E);
    if (!rc) rc = make_table(S, S->d.t_fp, cap_p, caps + 0, S->an_stream);
    if (!rc) rc = make_table(S, S->d.t_dd, cap_p, caps + 1, S->an_stream);
    if (!rc) rc = make_table(S, S->d.t_pend, cap_p, caps + 2, S->an_stream);
    if (!rc) rc = make_table(S, S->d.t_ep, cap_p, caps + 3, S->an_stream);
    if (!rc) rc = make_table(S, S->d.t_b, cap_b, caps + 4, S->an_stream);
    if (!rc) rc = make_table(S, S->d.t_pair, cap_p, caps + 5, S->an_stream);
    if (!rc) rc = make_table(S, S->d.t_rid, cap_p, caps + 6, S->an_stream);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.rid_open, 4ull * (cap_p + 1));
    if (!rc) rc = alloc_dev(S, (void**)&S->d.rid_wait, 4ull * (cap_p + 1));
    if (!rc) rc = alloc_dev(S, (void**)&S->d.wait_next, 4 * E);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.wait_del, 4 * E);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.kmax, 8 * SRV_NDEV);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.pend[0], 8ull * pend_cap);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.pend[1], 8ull * pend_cap);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.npend, 16);
    S->d.pend_cap = pend_cap;
    if (!rc) rc = make_table(S, S->d.t_ut, cap_p, caps + 7, S->an_stream);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.kcnt, 4 * SRV_NDEV);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.useg, 4 * E);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.utf[0], 8ull * pend_cap);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.utf[1], 8ull * pend_cap);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.utopen[0], 4ull * pend_cap);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.utopen[1], 4ull * pend_cap);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.nut, 32);
    if (!rc) rc = alloc_dev(S, (void**)&S->d.cur, 16);
    if (!rc) rc = alloc_dev(S, (void**)&S->fl.find, sizeof(odp_finding) * find_cap);
    if (!rc) rc = alloc_dev(S, (void**)&S->fl.complete, 8 * find_cap);
    if (!rc) rc = alloc_dev(S, (void**)&S->fl.nfind, 16);
    if (rc) return fail(rc);
    cudaMemsetAsync(S->d.kmax, 0, 8 * SRV_NDEV, S->an_stream);
    cudaMemsetAsync(S->d.gtail, 0xFF, 4 * E, S->an_stream);
    cudaMemsetAsync(S->d.rid_open, 0, 4ull * (cap_p + 1), S->an_stream);
    cudaMemsetAsync(S->d.rid_wait, 0xFF, 4ull * (cap_p + 1), S->an_stream);
    cudaMemsetAsync(S->d.rt_done, 0, E, S->an_stream);
    cudaMemsetAsync(S->d.npend, 0, 16, S->an_stream);
    cudaMemsetAsync(S->d.kcnt, 0, 4 * SRV_NDEV, S->an_stream);
    cudaMemsetAsync(S->d.nut, 0, 32, S->an_stream);
    cudaMemsetAsync(S->d.cur, 0, 16, S->an_stream);
    if (cudaHostAlloc((void**)&S->h_fl_find, sizeof(odp_finding) * find_cap, 0) != cudaSuccess ||
        cudaHostAlloc((void**)&S->h_fl_n, 16, 0) != cudaSuccess)
        return fail(ODP_ERR_OOM);
    S->slots.resize(cfg->n_slots);
    for (auto& sl : S->slots) {
        SlotDev& d = sl.d;
        rc = alloc_dev(S, (void**)&d.ev, sizeof(odp_event) * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.ptrs, 8 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.sizes, 8 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.fp, 16 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.xpos, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.fpos, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.par, sizeof(BatchPar));
        if (!rc) {
            d.nx = &d.par->nx;
            d.sort.hlen = &d.par->hlen;
        }
        if (!rc) rc = alloc_dev(S, (void**)&d.sfp, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.sdd, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.sb, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.skeys, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.svals, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.sort.keys_alt, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.sort.vals_alt, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.sort.hist, 4 * prim::sort_hist_words((uint32_t)B));
        if (!rc) {
            const size_t words = prim::scan_tmp_words(256u * ((uint32_t)B / prim::SORT_TILE + 2)) + 16;
            rc = alloc_dev(S, (void**)&d.sort.scan_tmp, 4 * words);
            if (!rc) cudaMemsetAsync(d.sort.scan_tmp, 0, 4 * words, S->an_stream);  // scans need it zero once
        }
        if (!rc) rc = alloc_dev(S, (void**)&d.find, sizeof(odp_finding) * find_cap);
        if (!rc) rc = alloc_dev(S, (void**)&d.complete, 8 * find_cap);
        if (!rc) rc = alloc_dev(S, (void**)&d.nfind, 16);
        if (!rc) rc = alloc_dev(S, (void**)&d.pa, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.pd, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.dalloc, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.rslot, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.bk, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.bktmp, 4 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.end1, 8 * B);
        if (!rc) rc = alloc_dev(S, (void**)&d.kst, 4 * 256);
        if (!rc) rc = alloc_dev(S, (void**)&d.kcn, 4 * 256);
        if (!rc) rc = alloc_dev(S, (void**)&d.cnt, 16);
        if (rc) return fail(rc);
        if (cudaHostAlloc((void**)&sl.h_ev, sizeof(odp_event) * B, 0) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_ptrs, 8 * B, 0) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_sizes, 8 * B, 0) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_xpos, 4 * B, 0) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_fpos, 4 * B, 0) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_par, sizeof(BatchPar), 0) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_find, sizeof(odp_finding) * find_cap, 0) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_complete, 8 * find_cap, 0) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_nfind, 16, 0) != cudaSuccess)
            return fail(ODP_ERR_OOM);
        if (cudaStreamCreateWithFlags(&sl.fp_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.fp_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.an_done, cudaEventDisableTiming) != cudaSuccess)
            return fail(ODP_ERR_CUDA);
        if ((rc = capture_analysis(S, sl)) != ODP_OK) return fail(rc);
    }
    S->small_ok = cudaFuncSetAttribute(srv_batch_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)prim::small_sort_smem(SRV_SMALL_BATCH)) == cudaSuccess;
    if (!S->small_ok) cudaGetLastError();
    if (cudaStreamSynchronize(S->an_stream) != cudaSuccess) return fail(ODP_ERR_CUDA);
    if ((rc = warm_up(S)) != ODP_OK) return fail(rc);
    S->submit_ns.assign(E, 0);
    S->latencies.reserve(E);  // no reallocation (under mu) while serving
    S->queue_lat.reserve(E);
    S->origin_prod.assign(E, 0);
    S->origin_seq.assign(E, 0);
    S->batcher = std::thread(odp::batcher_main, S);
    *out = S;
    return ODP_OK;
}

namespace {
// The calling thread's producer, registering it if needed.  A thread's id
// can be reused by a later thread once it has exited; the serial in its
// thread-local storage cannot, so a new thread never inherits an old
// producer's state.  The last server seen is cached per thread.
int producer_of_thread(odp_server* S, odp::Producer** out) {
    static std::atomic<uint64_t> next_serial{1};
    thread_local const uint64_t id = next_serial.fetch_add(1);
    thread_local uint64_t cached_server = 0;
    thread_local odp::Producer* cached = nullptr;
    if (cached_server == S->serial) {
        *out = cached;
        return ODP_OK;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    uint32_t p;
    auto it = S->producer_of.find(id);
    if (it != S->producer_of.end()) {
        p = it->second;
    } else {
        p = S->n_producers.load(std::memory_order_relaxed);
        if (p >= S->cfg.max_producers) return ODP_ERR_UNSUPPORTED;
        S->producer_of[id] = p;
        S->n_producers.store(p + 1, std::memory_order_release);
    }
    cached_server = S->serial;
    cached = &S->producers[p];
    *out = cached;
    return ODP_OK;
}
}  // namespace

int odp_server_attach(odp_server* S, uint64_t start_t_ns) {
    if (!S) return ODP_ERR_INVALID_ARG;
    odp::Producer* pr;
    int rc = producer_of_thread(S, &pr);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(pr->mu);
    pr->last_t = std::max(pr->last_t, start_t_ns);
    pr->last_seen = odp::now_ns();
    return ODP_OK;
}

int odp_server_begin(odp_server* S, uint64_t* t_start_ns) {
    if (!S || !t_start_ns) return ODP_ERR_INVALID_ARG;
    odp::Producer* pr;
    int rc = producer_of_thread(S, &pr);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(pr->mu);
    const uint64_t now = odp::now_ns();
    const uint64_t t = std::max(now, pr->last_t);
    pr->open.insert(t);
    pr->announces = true;
    pr->last_seen = now;
    *t_start_ns = t;
    return ODP_OK;
}

int odp_server_cancel(odp_server* S, uint64_t t_start_ns) {
    if (!S) return ODP_ERR_INVALID_ARG;
    odp::Producer* pr;
    int rc = producer_of_thread(S, &pr);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(pr->mu);
    auto it = pr->open.find(t_start_ns);
    if (it == pr->open.end()) return ODP_ERR_INVALID_ARG;
    pr->open.erase(it);
    pr->last_seen = odp::now_ns();
    return ODP_OK;
}

int odp_server_submit(odp_server* S, const odp_event* ev, const void* const* payloads,
                      uint64_t n) {
    if (!S || (n && (!ev || !payloads))) return ODP_ERR_INVALID_ARG;
    if (n == 0) return ODP_OK;
    const uint64_t t = odp::now_ns();
    odp::Producer* pr;
    int rc = producer_of_thread(S, &pr);
    if (rc) return rc;
    // reserve log capacity
    uint64_t cur = S->submitted.load();
    do {
        if (cur + n > S->cfg.max_events) return ODP_ERR_UNSUPPORTED;
    } while (!S->submitted.compare_exchange_weak(cur, cur + n));
    uint64_t zero = 0;
    S->first_submit.compare_exchange_strong(zero, t);
    std::lock_guard<std::mutex> lk(pr->mu);
    for (uint64_t i = 0; i < n; ++i) {
        odp::Pending q;
        q.ev = ev[i];
        q.payload = payloads[i];
        q.submit_ns = t;
        q.seq = pr->seq++;
        pr->last_t = std::max(pr->last_t, ev[i].t_start_ns);
        pr->q.push_back(q);
        // closes the latest open event that starts no later than this one
        auto it = pr->open.upper_bound(ev[i].t_start_ns);
        if (it != pr->open.begin()) pr->open.erase(std::prev(it));
    }
    pr->last_seen = t;
    return ODP_OK;
}

int odp_server_poll(odp_server* S, odp_finding* out, uint64_t cap, uint64_t* n_out) {
    if (!S || !n_out || (cap && !out)) return ODP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    uint64_t k = 0;
    while (k < cap && !S->outq.empty()) {
        out[k++] = S->outq.front();
        S->outq.pop_front();
    }
    *n_out = k;
    return S->error;
}

int odp_server_flush(odp_server* S) {
    if (!S) return ODP_ERR_INVALID_ARG;
    S->flushing = true;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::minutes(10);
        while (S->n_done < S->submitted) {
            if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
                S->flushing = false;
                return ODP_ERR_TIMEOUT;
            }
        }
    }
    // end of the trace: Alg. 4 for the pairs still waiting and the allocations
    // still open (their findings carry no latency)
    {
        std::lock_guard<std::mutex> an_lk(S->an_mu);
        cudaSetDevice(S->cfg.device);
        cudaStream_t as = S->an_stream;
        // pending decisions of Alg. 4 and 5 (one round), then the round trips of
        // groups with more than two endpoints, in rounds until none is dropped
        const uint32_t grid_mx =
            (unsigned)std::min<uint64_t>(1024, (std::max<uint64_t>(S->n_done, 1) + 255) / 256);
        const uint64_t max_rounds = S->cfg.max_events / std::max<uint32_t>(S->find_cap, 1) + 2;
        for (uint64_t round = 0; round <= max_rounds; ++round) {
            odp::srv_zero<<<1, 1, 0, as>>>(S->fl.nfind);
            if (round == 0)
                odp::srv_flush<<<256, 256, 0, as>>>(S->d, S->fl, S->find_cap, S->cfg.max_events);
            else
                odp::srv_mx_flush<<<grid_mx, 256, 0, as>>>(S->d, S->fl, S->find_cap, S->n_done,
                                                           S->cfg.max_events);
            cudaMemcpyAsync(S->h_fl_n, S->fl.nfind, 4, cudaMemcpyDeviceToHost, as);
            if (cudaStreamSynchronize(as) != cudaSuccess) {
                S->error = ODP_ERR_CUDA;
                break;
            }
            const uint32_t tried = *S->h_fl_n, n = std::min(tried, S->find_cap);
            cudaMemcpyAsync(S->h_fl_find, S->fl.find, sizeof(odp_finding) * n,
                            cudaMemcpyDeviceToHost, as);
            if (cudaStreamSynchronize(as) != cudaSuccess) {
                S->error = ODP_ERR_CUDA;
                break;
            }
            {
                std::lock_guard<std::mutex> lk(S->mu);
                for (uint32_t j = 0; j < n; ++j) S->outq.push_back(S->h_fl_find[j]);
                S->streamed += n;
                if (round == 0) S->find_overflow += tried - n;
            }
            if (round > 0 && tried <= S->find_cap) break;  // nothing dropped: done
            if (round == max_rounds) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->find_overflow += tried - n;
            }
        }
        odp::srv_flush_reset<<<1, 1, 0, as>>>(S->d);
        if (cudaStreamSynchronize(as) != cudaSuccess) S->error = ODP_ERR_CUDA;
    }
    S->flushing = false;
    return S->error;
}

int odp_server_log(odp_server* S, const odp_event** dev_log, uint64_t* n) {
    if (!S || !dev_log || !n) return ODP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *dev_log = S->d.log;
    *n = S->n_done;
    return ODP_OK;
}

int odp_server_origin(odp_server* S, uint32_t* producer, uint64_t* seq, uint64_t n) {
    if (!S || !producer || !seq) return ODP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (n > S->n_log) return ODP_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < n; ++i) {
        producer[i] = S->origin_prod[i];
        seq[i] = S->origin_seq[i];
    }
    return ODP_OK;
}

int odp_server_stats_get(odp_server* S, odp_server_stats* st) {
    if (!S || !st) return ODP_ERR_INVALID_ARG;
    std::vector<uint64_t> lat, qlat;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        st->events_submitted = S->submitted.load();
        st->events_processed = S->n_done;
        st->batches = S->batches;
        st->findings_streamed = S->streamed;
        st->late_events = S->late.load();
        st->first_submit_ns = S->first_submit.load();
        st->last_done_ns = S->last_done;
        lat = S->latencies;
        qlat = S->queue_lat;
    }
    std::sort(lat.begin(), lat.end());
    std::sort(qlat.begin(), qlat.end());
    auto pct = [](const std::vector<uint64_t>& v, double q) -> uint64_t {
        if (v.empty()) return 0;
        size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
        return v[std::min(i, v.size() - 1)];
    };
    st->latency_p50_ns = pct(lat, 0.50);
    st->latency_p99_ns = pct(lat, 0.99);
    st->latency_max_ns = lat.empty() ? 0 : lat.back();
    st->queue_p50_ns = pct(qlat, 0.50);
    st->queue_p99_ns = pct(qlat, 0.99);
    // groups with more than two endpoints (counted on the device table), and
    // findings or waiting decisions that did not fit
    st->rt_groups_at_flush = 0;
    st->device_bytes = S->dev_bytes;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        cudaSetDevice(S->cfg.device);
        uint32_t lost[2] = {0, 0};
        if (cudaMemcpy(&lost[0], S->d.npend + 2, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&lost[1], S->d.nut + 4, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return ODP_ERR_CUDA;
        st->stream_overflow = S->find_overflow + lost[0] + lost[1];
        if (S->n_done > 0 && S->d.t_ep.slots) {
            const uint32_t cap = S->d.t_ep.cap_max;
            std::vector<odp::prim::Slot> v((size_t)cap + 1);
            if (cudaMemcpy(v.data(), S->d.t_ep.slots, sizeof(odp::prim::Slot) * (cap + 1),
                           cudaMemcpyDeviceToHost) == cudaSuccess)
                for (const auto& x : v)
                    if (x.v != odp::prim::NONE32 && (x.v & odp::EP_MORE)) ++st->rt_groups_at_flush;
        }
    }
    return ODP_OK;
}

int odp_server_destroy(odp_server* S) {
    if (!S) return ODP_ERR_INVALID_ARG;
    S->stop = true;
    S->flushing = true;
    if (S->batcher.joinable()) S->batcher.join();
    cudaSetDevice(S->cfg.device);
    if (S->an_stream) cudaStreamSynchronize(S->an_stream);
    for (auto& sl : S->slots) {
        if (sl.fp_stream) {
            cudaStreamSynchronize(sl.fp_stream);
            odp::release_slot(odp::SLOT_FP_PLAN, sl.fp_stream);
            cudaStreamSynchronize(sl.fp_stream);
            cudaStreamDestroy(sl.fp_stream);
        }
        if (sl.fp_done) cudaEventDestroy(sl.fp_done);
        if (sl.an_done) cudaEventDestroy(sl.an_done);
        if (sl.an_graph) cudaGraphExecDestroy(sl.an_graph);
        for (void* h : {(void*)sl.h_ev, (void*)sl.h_ptrs, (void*)sl.h_sizes, (void*)sl.h_xpos,
                        (void*)sl.h_fpos, (void*)sl.h_par, (void*)sl.h_find, (void*)sl.h_complete,
                        (void*)sl.h_nfind})
            if (h) cudaFreeHost(h);
    }
    if (S->h_fl_find) cudaFreeHost(S->h_fl_find);
    if (S->h_fl_n) cudaFreeHost(S->h_fl_n);
    for (void* p : S->dev_blocks) cudaFree(p);
    if (S->an_stream) cudaStreamDestroy(S->an_stream);
    delete S;
    return ODP_OK;
}

}  // extern "C"
