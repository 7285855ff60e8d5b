// analyze.cu -- odp_analyze: Algorithms 1-5 of the paper (Sec. 5) as
// data-parallel GPU passes over the event log.
//
//   validate   record checks, order check, class of every event, lists of
//              transfers (X), alloc/deletes (P), kernels (K), to-device (U)
//   Alg. 1/2   table <fingerprint> -> content group key (the transfer whose
//              insert placed the fingerprint); stable sort of X by it.  The group
//              head and the start of the group's second run give each
//              destination's first receiver; every later transfer to it is a
//              duplicate.  With two endpoints in a content group the literal
//              queue walk reduces to "the first later reception at the
//              transfer's source", i.e. the start of the next run of equal
//              destinations; groups with more endpoints: sort by (group,
//              destination), per-endpoint "all receptions succeeded" in order
//              of last reception, partners by binary search
//   pairs      table <device, device address> -> dense id; stable sort of P;
//              alternating groups pair each ALLOC with the next DELETE, other
//              groups replay the nearest-open-ALLOC rule with a stack
//   Alg. 3     table <host address, device, bytes> -> first pair's alloc
//   kernels    stable sort of K by device; running maximum of kernel ends
//   Alg. 4     binary search of the first kernel whose running-max end
//              reaches the allocation's start (the literal monotone pointer)
//   Alg. 5     same search per to-device transfer; transfers after the last
//              kernel, barriers (overlapping the kernel) and candidates;
//              candidates sorted stably by host-address id, each member
//              overwritten by the next one of its segment
//   emit       per-kind ballot compaction in event order, wasted bytes/ns,
//              per-site rows, union of wasted events, summary
#include <algorithm>

#include "common.cuh"
#include "prims.cuh"

namespace odp {
namespace {

using prim::Key128;
using prim::NONE32;

constexpr uint32_t NOPART = 0xFFFFFFFEu;  // flagged without a partner
constexpr unsigned long long NO_ERR = ~0ull;
constexpr int NDEV = 129;                  // host + devices 0..127
constexpr int TPB = 256;

struct Hdr {
    unsigned long long err;
    unsigned long long t_end_max;
    unsigned long long saved_ns;
    unsigned long long unmatched;
    unsigned long long n_allocs, n_deletes, n_pairs;  // pairs counted where they are matched
    unsigned long long count[6], bytes[6], ns[6];
    uint32_t nX, nP, nK, nU;
    uint32_t nseg, nrun, nseg2, nsegU;
    uint32_t nB, nsegB;  // transfers / endpoint segments of groups with > 2 endpoints
    uint32_t any_bad;    // some content group has more than two endpoints
    uint32_t k_mixed, u_mixed;  // kernels / to-device transfers on more than one device
    uint32_t k_sortn, u_sortn;  // entries their by-device sorts move (0: one device, in order)
    uint32_t mx_n;       // transfers the multi-endpoint path scans: nX if any_bad, else 0
    uint32_t nA;         // allocations (at most this many pairs go into the Alg. 3 table)
    uint32_t scan_fault; // a scan's bounded wait gave up (reported as ODP_ERR_TIMEOUT)
    uint32_t total_findings, n_site_rows;
    uint32_t tcap;
    uint32_t n_gid_p, n_gid_u;  // distinct (device, device address) / candidate host-address keys
};

// Event field access (64-byte records).
struct Ev {
    const uint8_t* p;
    __device__ __forceinline__ uint64_t u64(uint32_t i, int off) const {
        return *(const uint64_t*)(p + 64ull * i + off);
    }
    __device__ __forceinline__ uint64_t t0(uint32_t i) const { return u64(i, 0); }
};

// Dense copies of the record fields the later passes read, one entry per
// event, written by k_validate (which reads every record anyway).  A pass over
// a list gathers 8-16 bytes per entry from them instead of a whole 128-byte
// line of records per entry.
struct EvCols {
    uint4* tt;        // {t_start, t_end}
    uint4* hd;        // {host_addr, dev_addr}
    uint64_t* bytes;  // bytes
    uint4* fp;        // {fp_lo, fp_hi} (dense: one DRAM fetch serves several transfers)
    uint32_t* site;   // site_id
};

__device__ __forceinline__ uint64_t lo64(uint4 v) { return ((uint64_t)v.y << 32) | v.x; }
__device__ __forceinline__ uint64_t hi64(uint4 v) { return ((uint64_t)v.w << 32) | v.z; }

// cls word: kind | (src + 1) << 8 | (dst + 1) << 16
__device__ __forceinline__ uint32_t c_kind(uint32_t c) { return c & 0xFF; }
__device__ __forceinline__ uint32_t c_src(uint32_t c) { return (c >> 8) & 0xFF; }
__device__ __forceinline__ uint32_t c_dst(uint32_t c) { return (c >> 16) & 0xFF; }

struct A {
    Ev ev;
    EvCols col;
    uint32_t n;
    uint32_t pack_alloc;  // slot keys leave bit 31 free: it carries "is ALLOC" through the pairs sort
    Hdr* h;
    uint32_t* cls;
    uint32_t *X, *P, *K, *U;
    uint2* drt;  // per event: .x the Alg. 1 partner, .y the Alg. 2 partner (one 8-byte word)
    uint32_t *ra, *ua, *ut, *del_of;
    uint32_t* wbits;      // wasted events, one bit per event
    uint8_t* bad;
    uint32_t *slot, *sk, *sv, *k2, *v2, *f1, *f2, *id1, *id2, *H, *R, *stk;
    uint32_t *pq;
    uint8_t* uc;
    uint64_t *ks, *ke;    // kernels sorted by device: start, running max of end
    uint32_t *dstart, *dend;  // kernel ranges per device, indexed by device number + 1
    unsigned long long* sites;  // [5][65536][3]
    prim::SplitTable tab;  // keys, then values: Alg. 3's first allocations
    prim::KeyTable ktab;   // the same memory as tab, keys only: contents, pairs, Alg. 5
    uint32_t* gid;         // per ktab slot: the dense group id of its key (tab's value array,
                           // which holds nothing before Alg. 3 or after it)
    odp_findings out;
};

__device__ __forceinline__ bool failed(const A& a) { return a.h->err != NO_ERR; }

// (n is read once: a device-side count re-read after every store would put
// its load on each iteration's path)
#define GRID_STRIDE(i, n)                                                          \
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x, i##_end = (n); i < i##_end; \
         i += gridDim.x * blockDim.x)


// ------------------------------------------------------------ validate

// Record checks on the fields of one event (loaded as three 16-byte words).
__device__ __forceinline__ bool record_ok(uint64_t t0, uint64_t t1, uint64_t by, uint32_t site,
                                          uint32_t w, uint32_t& cls) {
    const int kind = w & 0xFF;
    const int src = (int8_t)((w >> 8) & 0xFF), dst = (int8_t)((w >> 16) & 0xFF);
    cls = (uint32_t)kind | ((uint32_t)(src + 1) & 0xFF) << 8 | ((uint32_t)(dst + 1) & 0xFF) << 16;
    if (t1 < t0 || site >= ODP_MAX_SITES || by >= ODP_MAX_BYTES) return false;
    switch (kind) {
        case ODP_TO_DEV: return by > 0 && src == -1 && dst >= 0;
        case ODP_FROM_DEV: return by > 0 && src >= 0 && dst == -1;
        case ODP_DEV_TO_DEV: return by > 0 && src >= 0 && dst >= 0 && src != dst;
        case ODP_ALLOC:
        case ODP_DELETE:
        case ODP_KERNEL: return dst >= 0;
        default: return false;
    }
}

// One warp per 32-event chunk: record checks, order check, class word,
// per-(list, chunk) counts for the four lists.
__global__ void __launch_bounds__(TPB) k_validate(A a, uint32_t* ccnt, uint32_t nch) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long tmax = 0;
    uint32_t nallocs = 0, ndels = 0;
    for (uint32_t c = gw; c < nch; c += nw) {
        const uint32_t i = c * 32 + lane;
        const bool valid = i < a.n;
        uint64_t t0 = 0;
        uint4 q0 = make_uint4(0, 0, 0, 0), q1 = q0, q2 = q0, q3 = q0;
        if (valid) {
            const uint4* r = reinterpret_cast<const uint4*>(a.ev.p + 64ull * i);
            q0 = __ldg(r);
            q1 = __ldg(r + 1);
            q2 = __ldg(r + 2);
            q3 = __ldg(r + 3);
            t0 = ((uint64_t)q0.y << 32) | q0.x;
            a.col.tt[i] = q0;
            a.col.hd[i] = q1;
            a.col.bytes[i] = lo64(q2);
            a.col.fp[i] = make_uint4(q2.z, q2.w, q3.x, q3.y);
            a.col.site[i] = q3.z;
        }
        // start time of the previous event: the neighbour lane's, or a load
        uint64_t prev = __shfl_up_sync(ODP_FULL_MASK, t0, 1);
        uint32_t kd = 0;
        if (valid) {
            if (lane == 0 && i > 0) prev = a.ev.t0(i - 1);
            const uint64_t t1 = ((uint64_t)q0.w << 32) | q0.z;
            const uint64_t by = ((uint64_t)q2.y << 32) | q2.x;
            uint32_t cl;
            if (!record_ok(t0, t1, by, q3.z, q3.w, cl)) {
                record_error(&a.h->err, i, ODP_ERR_MALFORMED);
                cl = 0;
            } else if (i > 0 && t0 < prev) {
                record_error(&a.h->err, i, ODP_ERR_UNSORTED);
            }
            a.cls[i] = cl;
            kd = c_kind(cl);
            nallocs += kd == ODP_ALLOC;
            ndels += kd == ODP_DELETE;
            tmax = max(tmax, (unsigned long long)t1);
        }
        const uint32_t bx = __ballot_sync(ODP_FULL_MASK, kd == ODP_TO_DEV || kd == ODP_FROM_DEV ||
                                                             kd == ODP_DEV_TO_DEV);
        const uint32_t bp = __ballot_sync(ODP_FULL_MASK, kd == ODP_ALLOC || kd == ODP_DELETE);
        const uint32_t bk = __ballot_sync(ODP_FULL_MASK, kd == ODP_KERNEL);
        const uint32_t bu = __ballot_sync(ODP_FULL_MASK, kd == ODP_TO_DEV);
        if (lane == 0) {
            ccnt[0 * nch + c] = __popc(bx);
            ccnt[1 * nch + c] = __popc(bp);
            ccnt[2 * nch + c] = __popc(bk);
            ccnt[3 * nch + c] = __popc(bu);
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        tmax = max(tmax, __shfl_xor_sync(ODP_FULL_MASK, tmax, d));
        nallocs += __shfl_xor_sync(ODP_FULL_MASK, nallocs, d);
        ndels += __shfl_xor_sync(ODP_FULL_MASK, ndels, d);
    }
    if (lane == 0) {
        atomicMax(&a.h->t_end_max, tmax);
        if (nallocs) atomicAdd(&a.h->n_allocs, (unsigned long long)nallocs);
        if (ndels) atomicAdd(&a.h->n_deletes, (unsigned long long)ndels);
    }
}

// list lengths from the scanned chunk counts (scan covers 4 * nch)
__global__ void k_list_lengths(A a, const uint32_t* scanned, const uint32_t* total, uint32_t nch) {
    pdl_entry();
    if (threadIdx.x != 0) return;
    a.h->nX = scanned[1 * nch] - scanned[0];
    a.h->nP = scanned[2 * nch] - scanned[1 * nch];
    a.h->nK = scanned[3 * nch] - scanned[2 * nch];
    a.h->nU = *total - scanned[3 * nch];
    a.h->nA = (uint32_t)a.h->n_allocs;
}

// Stable compaction of event indices into the four lists, a warp per chunk.
// Four consecutive u32 from a 16-byte-aligned array (i0 % 4 == 0); entries at
// or past n read as `fill`.
__device__ __forceinline__ uint4 load4(const uint32_t* p, uint32_t i0, uint32_t n, uint32_t fill) {
    if (i0 + 4 <= n) return __ldg(reinterpret_cast<const uint4*>(p + i0));
    uint4 v = make_uint4(fill, fill, fill, fill);
    if (i0 < n) v.x = p[i0];
    if (i0 + 1 < n) v.y = p[i0 + 1];
    if (i0 + 2 < n) v.z = p[i0 + 2];
    return v;
}

// A warp takes 128 events (four chunks), four consecutive ones per lane;
// each list's entries of the group are placed by a warp scan of the lanes'
// counts after the group's scanned chunk offset.
__global__ void __launch_bounds__(TPB) k_compact(A a, const uint32_t* scanned, uint32_t nch) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nq = (nch + 3) / 4;
    uint32_t* lists[4] = {a.X, a.P, a.K, a.U};
    for (uint32_t g = gw; g < nq; g += nw) {
        const uint32_t i0 = g * 128 + lane * 4;
        const uint4 cl = load4(a.cls, i0, a.n, 0);
        const uint32_t kd[4] = {c_kind(cl.x), c_kind(cl.y), c_kind(cl.z), c_kind(cl.w)};
#pragma unroll
        for (int L = 0; L < 4; ++L) {
            bool pred[4];
            uint32_t cnt = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t k = i0 + j < a.n ? kd[j] : 0u;
                pred[j] = L == 0   ? k == ODP_TO_DEV || k == ODP_FROM_DEV || k == ODP_DEV_TO_DEV
                          : L == 1 ? k == ODP_ALLOC || k == ODP_DELETE
                          : L == 2 ? k == ODP_KERNEL
                                   : k == ODP_TO_DEV;
                cnt += pred[j];
            }
            uint32_t incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(ODP_FULL_MASK, incl, o);
                if (lane >= o) incl += t;
            }
            uint32_t pos = scanned[L * nch + 4 * g] - scanned[L * nch] + incl - cnt;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (pred[j]) lists[L][pos++] = i0 + j;
        }
    }
}

// ----------------------------------------------------- Alg. 1 (and ids)

// Group keys start as table slot indices: one slot per distinct key.  The
// pairs and Alg. 5 tables then replace each slot by a dense id numbered by
// the insert that put its key there (k_gid_keys), so the sorts that group
// equal keys (in an order of groups that nothing depends on) need only the
// bits of the number of distinct keys -- usually far fewer than the slots'.
// A full table cannot occur (capacity >= 1.25 x count); it would be
// reported, not mis-grouped.
__device__ __forceinline__ uint32_t slot_key(const A& a, uint32_t s, uint32_t e) {
    if (s == NONE32) record_error(&a.h->err, e, ODP_ERR_UNSUPPORTED);
    return s;
}

// Content groups are keyed by the event whose insert put the fingerprint
// into the table (the all-ones fingerprint, which has a slot of its own, by
// its first event): one store per content instead of a minimum kept per
// insert.  The inserting threads sweep the transfer list in time order, so
// the groups sort in nearly the order of their first transfers, and the
// passes that follow the sorted order touch the event-indexed arrays within
// a window that stays in L2.
// Four list entries per thread per step (spaced a grid apart, so the list
// loads and slot stores stay coalesced), their table probes in flight
// together.
constexpr int INS_B = 4;

#define BATCH_STRIDE(j0, n)                                                        \
    for (uint32_t j0 = blockIdx.x * blockDim.x + threadIdx.x; j0 < (n);            \
         j0 += INS_B * gridDim.x * blockDim.x)

__global__ void k_x_insert_fp(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t cap = *a.tab.cap_dev;
    const uint32_t n = a.h->nX, str = gridDim.x * blockDim.x;
    BATCH_STRIDE(j0, n) {
        uint32_t e[INS_B], out[INS_B];
        bool use[INS_B];
        Key128 key[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t j = j0 + b * str;
            use[b] = j < n;
            e[b] = use[b] ? a.X[j] : 0;
        }
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint4 f = use[b] ? a.col.fp[e[b]] : make_uint4(0, 0, 0, 0);
            key[b] = Key128{lo64(f), hi64(f)};
        }
        bool fresh[INS_B];
        prim::table_insert_batch<INS_B, false, true, false>(a.ktab, cap, key, e, use, out, fresh);
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            if (!use[b]) continue;
            if (fresh[b]) a.gid[out[b]] = e[b];
            else if (out[b] == a.ktab.cap_max) atomicMin(a.gid + out[b], e[b]);
            a.slot[j0 + b * str] = slot_key(a, out[b], e[b]);
        }
    }
}

__global__ void k_x_cid(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t n = a.h->nX, str = gridDim.x * blockDim.x;
    BATCH_STRIDE(j0, n) {
        uint32_t sl[INS_B], v[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) sl[b] = j0 + b * str < n ? a.slot[j0 + b * str] : NONE32;
#pragma unroll
        for (int b = 0; b < INS_B; ++b) v[b] = sl[b] != NONE32 ? a.gid[sl[b]] : 0;
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t j = j0 + b * str;
            if (j >= n) continue;
            a.sk[j] = v[b];
            a.sv[j] = a.X[j];
        }
    }
}

// ------------------------------------------------------------- Alg. 2

// Group and run heads; the class word of each sorted transfer is gathered
// once into a.k2 (in sorted order) for the passes that follow.
__global__ void k_rt_flags(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(q, a.h->nX) {
        const bool head = q == 0 || a.sk[q] != a.sk[q - 1];
        const uint32_t c = a.cls[a.sv[q]];
        const bool run = head || c_dst(c) != c_dst(a.cls[a.sv[q - 1]]);
        a.f1[q] = head;
        a.f2[q] = run;
        a.k2[q] = c;
    }
}

__global__ void k_rt_starts(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t n = a.h->nX, str = gridDim.x * blockDim.x;
    BATCH_STRIDE(q0, n) {
        uint32_t f1[INS_B], f2[INS_B], i1[INS_B], i2[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t q = q0 + b * str;
            const bool in = q < n;
            f1[b] = in ? a.f1[q] : 0u;
            f2[b] = in ? a.f2[q] : 0u;
            i1[b] = in ? a.id1[q] : 0u;
            i2[b] = in ? a.id2[q] : 0u;
        }
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t q = q0 + b * str;
            if (q >= n) continue;
            if (f1[b]) a.H[i1[b]] = q;
            if (f2[b]) a.R[i2[b]] = q;
            a.bad[q] = 0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.H[a.h->nseg] = n;
        a.R[a.h->nrun] = n;
    }
}

__device__ __forceinline__ bool same_endpoints(uint32_t c, uint32_t d) {
    const uint32_t s1 = c_src(c), d1 = c_dst(c), s2 = c_src(d), d2 = c_dst(d);
    return (s1 == s2 && d1 == d2) || (s1 == d2 && d1 == s2);
}

__global__ void k_rt_check(A a) {
    pdl_entry();
    if (failed(a)) return;
    __shared__ int blk_bad;
    if (threadIdx.x == 0) blk_bad = 0;
    __syncthreads();
    GRID_STRIDE(q, a.h->nX) {
        const uint32_t s = a.id1[q] + a.f1[q] - 1;
        const uint32_t h = a.H[s];
        if (!same_endpoints(a.k2[q], a.k2[h])) {
            a.bad[s] = 1;
            blk_bad = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk_bad) atomicOr(&a.h->any_bad, 1u);
}

// Two endpoints: a transfer pairs with the first event of the next run of
// its content group (the next run receives at the other endpoint, which is
// the transfer's source).  Alg. 1 comes from the same order: the first
// receiver of <content, destination> is the group head when the destination
// matches the head's, else the start of the group's second run.
__global__ void k_rt_partner(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t nrun = a.h->nrun;
    // the multi-endpoint passes that follow scan the transfers only if needed
    if (blockIdx.x == 0 && threadIdx.x == 0) a.h->mx_n = a.h->any_bad ? a.h->nX : 0u;
    GRID_STRIDE(q, a.h->nX) {
        const uint32_t s = a.id1[q] + a.f1[q] - 1;
        if (a.bad[s]) continue;
        const uint32_t e = a.sv[q];
        const uint32_t r = a.id2[q] + a.f2[q] - 1;
        uint32_t rt = NONE32;
        if (r + 1 < nrun) {
            const uint32_t q2 = a.R[r + 1];
            if (!a.f1[q2]) rt = a.sv[q2];
        }
        const uint32_t h = a.H[s];
        uint32_t first;
        if (c_dst(a.k2[q]) == c_dst(a.k2[h])) first = a.sv[h];
        else first = a.sv[a.R[a.id2[h] + 1]];
        // one write for both partners (the events scatter: one sector, not two)
        if (rt != NONE32 || first != e) a.drt[e] = make_uint2(first != e ? first : NONE32, rt);
    }
}

// ------------------------------------ Alg. 2 with more than two endpoints
//
// A content group (transfers of one content id, in time order) with three or
// more endpoints.  Alg. 2 keeps one queue per endpoint holding the group's
// receptions there; a transfer from A reports the front of A's queue if it is
// non-empty and then pops the queue of its own destination.  Without the
// queues: let last_A be A's last reception and allOK_A say that every
// reception at A succeeded (produced a finding).  Pops of A's queue before
// time t equal the successful receptions at A before t, so
//   * a transfer from A at t succeeds iff t < last_A or not allOK_A (a source
//     that never receives has an empty queue: last = -1, allOK = true);
//   * its partner is the k-th reception at A, k = successful receptions at A
//     before t;
//   * a reception r from X is "late" when r > last_X, and it fails iff it is
//     late and allOK_X; so allOK_D = no late reception at D comes from an
//     endpoint X with allOK_X.  A late reception from X at D has
//     last_X < r <= last_D, so allOK is settled endpoint by endpoint in
//     increasing order of last.
// The passes: compact the groups' transfers, sort them stably by (group,
// destination) so each endpoint's receptions are one segment in time order;
// per reception, the source's segment (binary search) and the late flag,
// folded into a per-segment set of late sources; per group, the allOK
// recursion over its segments (endpoints <= 129, independent of the group's
// length); per reception, success; a scan of successes; per transfer, the
// partner by two binary searches.  Alg. 1 in these groups: the first element
// of each segment is the first receiver, the others are duplicates of it.

__device__ __forceinline__ uint32_t group_of(const A& a, uint32_t q) { return a.id1[q] + a.f1[q] - 1; }

// flags of the transfers in groups with more than two endpoints
__global__ void k_mx_flag(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(q, a.h->mx_n) a.f2[q] = a.bad[group_of(a, q)];
}

// compacted list: key = destination, value = position in content order
__global__ void k_mx_scatter(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(q, a.h->mx_n) {
        if (!a.f2[q]) continue;
        const uint32_t j = a.id2[q];
        a.k2[j] = c_dst(a.cls[a.sv[q]]);
        a.v2[j] = q;
    }
}

__global__ void k_mx_gkey(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(i, a.h->nB) a.k2[i] = group_of(a, a.v2[i]);
}

// Ld[i] = destination (in a.slot), segment heads (in a.f2), group starts.
__global__ void k_mx_heads(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(i, a.h->nB) {
        const uint32_t s = a.k2[i];
        const uint32_t d = c_dst(a.cls[a.sv[a.v2[i]]]);
        a.slot[i] = d;
        const bool ghead = i == 0 || a.k2[i - 1] != s;
        if (ghead) a.pq[s] = i;
        a.f2[i] = ghead || c_dst(a.cls[a.sv[a.v2[i - 1]]]) != d;
    }
}

// Segment starts (in a.R) and cleared per-segment late-source sets: a.ks/a.ke
// hold one 128-bit set per segment (endpoint codes 0..127); a.uc holds per
// segment bit 0 = late from code 128, bit 1 = allOK, bit 2 = late from an
// endpoint that never receives.
__global__ void k_mx_starts(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t nB = a.h->nB;
    uint4* mask = reinterpret_cast<uint4*>(a.ks);
    GRID_STRIDE(i, nB) {
        if (!a.f2[i]) continue;
        const uint32_t g = a.id2[i];
        a.R[g] = i;
        mask[g] = make_uint4(0, 0, 0, 0);
        a.uc[g] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.R[a.h->nsegB] = nB;
}

// Segment of endpoint x in group s (NONE32 if x never receives there).
__device__ __forceinline__ uint32_t mx_find(const A& a, uint32_t s, uint32_t x) {
    uint32_t lo = a.pq[s], hi = lo + (a.H[s + 1] - a.H[s]);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.slot[mid] < x) lo = mid + 1; else hi = mid;
    }
    if (lo < a.pq[s] + (a.H[s + 1] - a.H[s]) && a.slot[lo] == x) return a.id2[lo];
    return NONE32;
}

__device__ __forceinline__ uint32_t mx_last(const A& a, uint32_t g) { return a.v2[a.R[g + 1] - 1]; }

// Per reception: source segment (in a.stk) and the late flag, folded into the
// destination segment's set (one atomic per distinct (segment, source) of a
// warp).
__global__ void k_mx_late(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t nB = a.h->nB;
    const int lane = threadIdx.x & 31;
    uint32_t* mask = reinterpret_cast<uint32_t*>(a.ks);
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < nB;
         base += gridDim.x * blockDim.x) {
        const uint32_t i = base + lane;
        unsigned long long key = ~0ull;
        uint32_t x = 0, g = 0;
        bool late = false;
        if (i < nB) {
            const uint32_t q = a.v2[i];
            x = c_src(a.cls[a.sv[q]]);
            const uint32_t xs = mx_find(a, a.k2[i], x);
            a.stk[i] = xs;
            g = a.id2[i] + a.f2[i] - 1;
            late = xs == NONE32 || q > mx_last(a, xs);
            if (late) key = ((unsigned long long)g << 9) | (xs == NONE32 ? 256u : x);
        }
        const uint32_t peers = __match_any_sync(ODP_FULL_MASK, key);
        if (late && lane == __ffs(peers) - 1) {
            if ((key & 511u) == 256u) {
                atomicOr(reinterpret_cast<unsigned int*>(a.uc + (g & ~3u)), 4u << (8 * (g & 3u)));
            } else if (x == 128) {
                atomicOr(reinterpret_cast<unsigned int*>(a.uc + (g & ~3u)), 1u << (8 * (g & 3u)));
            } else {
                atomicOr(&mask[4ull * g + (x >> 5)], 1u << (x & 31));
            }
        }
    }
}

// Per group: allOK of its endpoints in increasing order of last reception.
__global__ void k_mx_ok(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t nseg = a.h->nseg;
    const uint4* mask = reinterpret_cast<const uint4*>(a.ks);
    GRID_STRIDE(s, nseg) {
        if (!a.bad[s]) continue;
        const uint32_t lo = a.pq[s], hi = lo + (a.H[s + 1] - a.H[s]);
        // segments [g0, g1): lo is a segment head, hi - 1 is in the last one
        const uint32_t g0 = a.id2[lo], g1 = a.id2[hi - 1] + a.f2[hi - 1];
        uint32_t ok[4] = {0, 0, 0, 0};
        bool ok128 = false;
        uint32_t done_below = 0;  // last position already processed
        bool any = false;
        for (uint32_t it = g0; it < g1; ++it) {
            // next segment: smallest last above the previous one (lasts are distinct)
            uint32_t best = NONE32, best_last = NONE32;
            for (uint32_t g = g0; g < g1; ++g) {
                const uint32_t l = mx_last(a, g);
                if ((!any || l > done_below) && l < best_last) {
                    best_last = l;
                    best = g;
                }
            }
            any = true;
            done_below = best_last;
            const uint4 m = mask[best];
            const uint32_t fl = a.uc[best];
            const bool all_ok = !(fl & 4u) && !((fl & 1u) && ok128) && !(m.x & ok[0]) &&
                                !(m.y & ok[1]) && !(m.z & ok[2]) && !(m.w & ok[3]);
            if (all_ok) {
                const uint32_t d = a.slot[a.R[best]];
                if (d == 128) ok128 = true;
                else ok[d >> 5] |= 1u << (d & 31);
                a.uc[best] = (uint8_t)(fl | 2u);
            }
        }
    }
}

// Per reception: success (in a.k2, scanned into a.sk next).
__global__ void k_mx_succ(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(i, a.h->nB) {
        const uint32_t xs = a.stk[i];
        bool fail = true;
        if (xs != NONE32) fail = a.v2[i] > mx_last(a, xs) && (a.uc[xs] & 2u);
        a.k2[i] = !fail;
    }
}

// Per transfer: Alg. 1 inside its segment, Alg. 2 partner.
__global__ void k_mx_partner(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(i, a.h->nB) {
        const uint32_t q = a.v2[i];
        const uint32_t e = a.sv[q];
        const uint32_t head = a.R[a.id2[i] + a.f2[i] - 1];
        if (head != i) a.drt[e].x = a.sv[a.v2[head]];
        const uint32_t xs = a.stk[i];
        if (xs == NONE32) continue;
        const uint32_t st = a.R[xs], en = a.R[xs + 1];
        if (!(q < a.v2[en - 1] || !(a.uc[xs] & 2u))) continue;
        uint32_t lo = st, hi = en;  // receptions at the source before q
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.v2[mid] < q) lo = mid + 1; else hi = mid;
        }
        // successes among [st, lo): a.k2 = success flags, a.sk = their exclusive scan
        const uint32_t k = lo == st ? 0 : a.sk[lo - 1] + a.k2[lo - 1] - a.sk[st];
        if (st + k < en) a.drt[e].y = a.sv[a.v2[st + k]];
    }
}

// ------------------------------------------------------------- pairs

__global__ void k_p_insert(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t cap = *a.ktab.cap_dev;
    const uint32_t n = a.h->nP, str = gridDim.x * blockDim.x;
    BATCH_STRIDE(j0, n) {
        uint32_t e[INS_B], out[INS_B];
        bool use[INS_B];
        Key128 key[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t j = j0 + b * str;
            use[b] = j < n;
            e[b] = use[b] ? a.P[j] : 0;
        }
        uint32_t flag[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t c = use[b] ? a.cls[e[b]] : 0;
            key[b] = use[b] ? Key128{hi64(a.col.hd[e[b]]), (uint64_t)c_dst(c)} : Key128{0, 0};
            flag[b] = a.pack_alloc && c_kind(c) == ODP_ALLOC ? 0x80000000u : 0u;
        }
        bool fresh[INS_B];
        prim::table_insert_batch<INS_B, false, true, false>(a.ktab, cap, key, e, use, out, fresh);
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            if (!use[b]) continue;
            // (a key's high half is a device number: never the all-ones key)
            if (fresh[b]) a.gid[out[b]] = atomicAdd(&a.h->n_gid_p, 1u) + 1u;
            a.sk[j0 + b * str] = slot_key(a, out[b], e[b]) | flag[b];
            a.sv[j0 + b * str] = e[b];
        }
    }
}

// Group heads of the sorted alloc/delete list, and whether each entry is an
// ALLOC into a.k2 (in sorted order): from bit 31 of the sort key where the
// sort carried it there, else gathered from the class words.
__global__ void k_seg_heads(A a, const uint32_t* count) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t m = a.pack_alloc ? 0x7FFFFFFFu : 0xFFFFFFFFu;
    GRID_STRIDE(q, *count) {
        const uint32_t k = a.sk[q];
        a.f1[q] = q == 0 || (k & m) != (a.sk[q - 1] & m);
        a.k2[q] = a.pack_alloc ? k >> 31 : c_kind(a.cls[a.sv[q]]) == ODP_ALLOC;
    }
}

__global__ void k_seg_starts(A a, const uint32_t* count, const uint32_t* nseg) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t n = *count;
    GRID_STRIDE(q, n) {
        if (a.f1[q]) a.H[a.id1[q]] = q;
        a.bad[q] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.H[*nseg] = n;
}

__device__ __forceinline__ bool is_alloc(const A& a, uint32_t e) {
    return c_kind(a.cls[e]) == ODP_ALLOC;
}

__global__ void k_p_check(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(q, a.h->nP) {
        const uint32_t s = a.id1[q] + a.f1[q] - 1;
        const uint32_t lo = a.H[s], hi = a.H[s + 1];
        const bool al = a.k2[q];
        bool bad;
        if (!al) bad = q == lo || !a.k2[q - 1];
        else bad = q + 1 < hi && a.k2[q + 1];
        if (bad) a.bad[s] = 1;
    }
}

__global__ void k_p_match(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t n = a.h->nP, str = gridDim.x * blockDim.x;
    uint32_t pairs = 0;
    BATCH_STRIDE(q0, n) {
        uint32_t sg[INS_B], e[INS_B], d[INS_B];
        bool al[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t q = q0 + b * str;
            al[b] = q < n && a.k2[q];
            sg[b] = al[b] ? a.id1[q] + a.f1[q] - 1 : 0u;
            e[b] = al[b] ? a.sv[q] : 0u;
            d[b] = al[b] && q + 1 < n ? a.sv[q + 1] : NONE32;
        }
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t q = q0 + b * str;
            // the next entry closes this ALLOC if it lies in the same group
            if (al[b] && !a.bad[sg[b]] && q + 1 < a.H[sg[b] + 1]) {
                a.del_of[e[b]] = d[b];
                ++pairs;
            }
        }
    }
    for (int k = 16; k > 0; k >>= 1) pairs += __shfl_xor_sync(ODP_FULL_MASK, pairs, k);
    if ((threadIdx.x & 31) == 0 && pairs) atomicAdd(&a.h->n_pairs, (unsigned long long)pairs);
}

// Non-alternating groups: a DELETE closes the nearest earlier open ALLOC.
__global__ void k_p_literal(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(s, a.h->nseg2) {
        if (!a.bad[s]) continue;
        const uint32_t lo = a.H[s], hi = a.H[s + 1];
        uint32_t depth = 0;
        unsigned long long unmatched = 0, pairs = 0;
        for (uint32_t q = lo; q < hi; ++q) {
            const uint32_t e = a.sv[q];
            if (is_alloc(a, e)) {
                a.stk[lo + depth++] = e;
            } else if (depth > 0) {
                a.del_of[a.stk[lo + --depth]] = e;
                ++pairs;
            } else {
                ++unmatched;
            }
        }
        if (unmatched) atomicAdd(&a.h->unmatched, unmatched);
        if (pairs) atomicAdd(&a.h->n_pairs, pairs);
    }
}

// ------------------------------------------------------------- Alg. 3

__global__ void k_ra_insert(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t cap = *a.tab.cap_dev;
    const uint32_t n = a.h->nP, str = gridDim.x * blockDim.x;
    BATCH_STRIDE(j0, n) {
        uint32_t e[INS_B], out[INS_B];
        bool use[INS_B], in[INS_B];
        Key128 key[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t j = j0 + b * str;
            in[b] = j < n;
            e[b] = in[b] ? a.P[j] : 0;
        }
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            use[b] = in[b] && is_alloc(a, e[b]) && a.del_of[e[b]] != NONE32;
            key[b] = use[b] ? Key128{lo64(a.col.hd[e[b]]),
                                     a.col.bytes[e[b]] | ((uint64_t)c_dst(a.cls[e[b]]) << 56)}
                            : Key128{0, 0};
        }
        prim::table_insert_batch<INS_B, true, true, true>(a.tab, cap, key, e, use, out);
#pragma unroll
        for (int b = 0; b < INS_B; ++b)
            if (in[b]) a.slot[j0 + b * str] = out[b];
    }
}

__global__ void k_ra_flag(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t n = a.h->nP, str = gridDim.x * blockDim.x;
    BATCH_STRIDE(j0, n) {
        uint32_t sl[INS_B], first[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) sl[b] = j0 + b * str < n ? a.slot[j0 + b * str] : NONE32;
#pragma unroll
        for (int b = 0; b < INS_B; ++b) first[b] = sl[b] != NONE32 ? a.tab.vals[sl[b]] : NONE32;
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            if (sl[b] == NONE32) continue;
            const uint32_t e = a.P[j0 + b * str];
            if (first[b] != e) a.ra[e] = first[b];
        }
    }
}

// ------------------------------------------------------------ kernels

// Device keys of a list in time order; *mixed is set when they are not all
// the device of the list's first entry.
__global__ void k_dev_keys(A a, const uint32_t* list, const uint32_t* count, uint32_t* mixed) {
    pdl_entry();
    if (failed(a)) return;
    __shared__ int blk_mixed;
    if (threadIdx.x == 0) blk_mixed = 0;
    __syncthreads();
    const uint32_t n = *count;
    const uint32_t d0 = n ? c_dst(a.cls[list[0]]) : 0u;
    GRID_STRIDE(j, n) {
        const uint32_t e = list[j];
        const uint32_t d = c_dst(a.cls[e]);
        a.sk[j] = d;
        a.sv[j] = e;
        if (d != d0) blk_mixed = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk_mixed) atomicOr(mixed, 1u);
}

// A list on one device is already sorted by device: its sort moves nothing.
__global__ void k_sort_count(const uint32_t* count, const uint32_t* mixed, uint32_t* sort_n) {
    pdl_entry();
    if (blockIdx.x == 0 && threadIdx.x == 0) *sort_n = *mixed ? *count : 0u;
}

__global__ void k_k_bounds(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t n = a.h->nK;
    GRID_STRIDE(q, n) {
        const uint32_t d = a.sk[q];
        if (q == 0 || a.sk[q - 1] != d) a.dstart[d] = q;
        if (q + 1 == n || a.sk[q + 1] != d) a.dend[d] = q + 1;
        const uint4 t = a.col.tt[a.sv[q]];
        a.ks[q] = lo64(t);
        a.ke[q] = hi64(t);
    }
}

// Running maximum of kernel ends within each device: one block per device,
// an inclusive max-scan per 1024-kernel tile with a carry between tiles.
constexpr int PMAX_THREADS = 1024;

__global__ void __launch_bounds__(PMAX_THREADS) k_k_pmax(A a) {
    pdl_entry();
    if (failed(a)) return;
    __shared__ unsigned long long wmax[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lo = a.dstart[blockIdx.x], hi = a.dend[blockIdx.x];
    unsigned long long carry = 0;
    for (uint32_t base = lo; base < hi; base += PMAX_THREADS) {
        const uint32_t q = base + threadIdx.x;
        unsigned long long v = q < hi ? a.ke[q] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(ODP_FULL_MASK, v, o);
            if (lane >= o) v = max(v, y);
        }
        if (lane == 31) wmax[warp] = v;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = wmax[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(ODP_FULL_MASK, w, o);
                if (lane >= o) w = max(w, y);
            }
            wmax[lane] = w;
        }
        __syncthreads();
        if (warp > 0) v = max(v, wmax[warp - 1]);
        if (q < hi) a.ke[q] = max(v, carry);
        carry = max(carry, wmax[31]);
        __syncthreads();
    }
}

// First kernel position p in [dstart, dend) of device d with running-max
// end >= t (dend if none): the monotone pointer of Alg. 4 and 5.
__device__ __forceinline__ uint32_t first_kernel(const A& a, uint32_t d, uint64_t t) {
    uint32_t lo = a.dstart[d], hi = a.dend[d];
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a.ke[mid] >= t) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// ------------------------------------------------------------- Alg. 4

__global__ void k_ua(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint64_t trace_end = a.h->t_end_max;
    const uint32_t n = a.h->nP, str = gridDim.x * blockDim.x;
    BATCH_STRIDE(j0, n) {
        uint32_t e[INS_B], c[INS_B], del[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) e[b] = j0 + b * str < n ? a.P[j0 + b * str] : NONE32;
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            c[b] = e[b] != NONE32 ? a.cls[e[b]] : 0;
            del[b] = e[b] != NONE32 ? a.del_of[e[b]] : NONE32;
        }
        uint64_t t0[INS_B], end[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const bool al = c_kind(c[b]) == ODP_ALLOC;
            t0[b] = al ? lo64(a.col.tt[e[b]]) : 0;
            end[b] = !al ? 0 : del[b] != NONE32 ? hi64(a.col.tt[del[b]]) : trace_end;
        }
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            if (c_kind(c[b]) != ODP_ALLOC) continue;
            const uint32_t d = c_dst(c[b]);  // device number + 1
            const uint32_t p = first_kernel(a, d, t0[b]);
            if (p == a.dend[d] || a.ks[p] > end[b]) a.ua[e[b]] = del[b] != NONE32 ? del[b] : NOPART;
        }
    }
}

// ------------------------------------------------------------- Alg. 5

__global__ void k_ut_class(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(q, a.h->nU) {
        const uint32_t e = a.sv[q];
        const uint32_t d = a.sk[q];  // device number + 1
        const uint64_t t = lo64(a.col.tt[e]);
        const uint32_t p = first_kernel(a, d, t);
        uint8_t c;
        if (p == a.dend[d]) {
            c = 2;                       // after the last kernel
            a.ut[e] = NOPART;
        } else if (a.ks[p] <= t) {
            c = 1;                       // overlaps kernel p: clears candidates
        } else {
            c = 0;                       // candidate
        }
        a.pq[q] = p;
        a.uc[q] = c;
    }
}

__global__ void k_ut_heads(A a) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(q, a.h->nU) {
        a.f1[q] = q == 0 || a.sk[q] != a.sk[q - 1] || a.pq[q] != a.pq[q - 1] || a.uc[q - 1] == 1;
    }
}

// Candidates grouped by host address (few distinct addresses: the table
// stays in L2); the group key is the address's slot (then its dense id),
// non-candidates get NONE32 (then 0).
__global__ void k_ut_insert(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t cap = *a.ktab.cap_dev;
    const uint32_t n = a.h->nU, str = gridDim.x * blockDim.x;
    BATCH_STRIDE(q0, n) {
        uint32_t e[INS_B], out[INS_B];
        bool use[INS_B];
        Key128 key[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t q = q0 + b * str;
            use[b] = q < n && a.uc[q] == 0;
            e[b] = use[b] ? a.sv[q] : 0;
            key[b] = use[b] ? Key128{lo64(a.col.hd[e[b]]), 1} : Key128{0, 0};
        }
        bool fresh[INS_B];
        prim::table_insert_batch<INS_B, false, true, false>(a.ktab, cap, key, e, use, out, fresh);
#pragma unroll
        for (int b = 0; b < INS_B; ++b) {
            const uint32_t q = q0 + b * str;
            if (q >= n) continue;
            // (a key's high half is 1: never the all-ones key)
            if (fresh[b]) a.gid[out[b]] = atomicAdd(&a.h->n_gid_u, 1u) + 1u;
            a.k2[q] = use[b] ? slot_key(a, out[b], e[b]) : NONE32;
            a.v2[q] = q;
        }
    }
}

// Slot keys to dense group ids, after the inserts: keys[q] = gid[slot], bit
// `flag` carried over; NONE32 (no slot) becomes 0.
__global__ void k_gid_keys(A a, uint32_t* keys, const uint32_t* count, uint32_t flag) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t n = *count, str = gridDim.x * blockDim.x;
    BATCH_STRIDE(q0, n) {
        uint32_t k[INS_B];
#pragma unroll
        for (int b = 0; b < INS_B; ++b) k[b] = q0 + b * str < n ? keys[q0 + b * str] : NONE32;
#pragma unroll
        for (int b = 0; b < INS_B; ++b) k[b] = k[b] == NONE32 ? 0u : a.gid[k[b] & ~flag] | (k[b] & flag);
#pragma unroll
        for (int b = 0; b < INS_B; ++b)
            if (q0 + b * str < n) keys[q0 + b * str] = k[b];
    }
}

// After the stable sort by host group, a candidate is overwritten by the
// next candidate of its group when both lie in the same segment.
__global__ void k_ut_next(A a) {
    pdl_entry();
    if (failed(a)) return;
    const uint32_t nU = a.h->nU;
    GRID_STRIDE(r, nU) {
        if (a.k2[r] == 0 || r + 1 >= nU || a.k2[r + 1] != a.k2[r]) continue;
        const uint32_t q = a.v2[r], q2 = a.v2[r + 1];
        const uint32_t s1 = a.id1[q] + a.f1[q] - 1, s2 = a.id1[q2] + a.f1[q2] - 1;
        if (s1 == s2) a.ut[a.sv[q]] = a.sv[q2];
    }
}

// ------------------------------------------------------------ emission

__device__ __forceinline__ uint64_t lohi(uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; }

__device__ __forceinline__ uint32_t partner_of(const A& a, int kind, uint32_t i) {
    switch (kind) {
        case ODP_DD: return a.drt[i].x;
        case ODP_RT: return a.drt[i].y;
        case ODP_RA: return a.ra[i];
        case ODP_UA: return a.ua[i];
        default: return a.ut[i];
    }
}

__device__ __forceinline__ const uint32_t* partner_array(const A& a, int kind) {
    switch (kind) {
        case ODP_RA: return a.ra;
        case ODP_UA: return a.ua;
        default: return a.ut;
    }
}


// Findings per (kind, 32-event chunk) from the partner arrays alone (the
// pairs are counted where they are matched).  A warp takes 128 events (four
// chunks), four per lane with 16-byte loads; lanes 8k..8k+7 sum chunk k.
__global__ void k_em_count(A a, uint32_t* wcnt, uint32_t nch) {
    pdl_entry();
    if (failed(a)) return;
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nq = (nch + 3) / 4;
    for (uint32_t g = gw; g < nq; g += nw) {
        const uint32_t i0 = g * 128 + lane * 4;
        const uint32_t c = g * 4 + (lane >> 3);
        // Alg. 1 and 2 partners of events i0..i0+3 (two 16-byte words of drt)
        uint4 p0 = make_uint4(NONE32, NONE32, NONE32, NONE32), p1 = p0;
        if (i0 + 4 <= a.n) {
            p0 = __ldg(reinterpret_cast<const uint4*>(a.drt + i0));
            p1 = __ldg(reinterpret_cast<const uint4*>(a.drt + i0 + 2));
        } else {
            if (i0 < a.n) p0.x = a.drt[i0].x, p0.y = a.drt[i0].y;
            if (i0 + 1 < a.n) p0.z = a.drt[i0 + 1].x, p0.w = a.drt[i0 + 1].y;
            if (i0 + 2 < a.n) p1.x = a.drt[i0 + 2].x, p1.y = a.drt[i0 + 2].y;
        }
#pragma unroll
        for (int kind = 1; kind <= 5; ++kind) {
            const uint4 v = kind == ODP_DD   ? make_uint4(p0.x, p0.z, p1.x, p1.z)
                            : kind == ODP_RT ? make_uint4(p0.y, p0.w, p1.y, p1.w)
                                             : load4(partner_array(a, kind), i0, a.n, NONE32);
            uint32_t k = (v.x != NONE32) + (v.y != NONE32) + (v.z != NONE32) + (v.w != NONE32);
            k += __shfl_xor_sync(ODP_FULL_MASK, k, 1);
            k += __shfl_xor_sync(ODP_FULL_MASK, k, 2);
            k += __shfl_xor_sync(ODP_FULL_MASK, k, 4);
            if ((lane & 7) == 0 && c < nch) wcnt[(kind - 1) * nch + c] = k;
        }
    }
}

// Site rows are accumulated per block in a shared-memory hash table of
// (kind, site) keys and flushed to the dense global table once per block;
// keys that do not fit go straight to global atomics.
constexpr int SITE_SLOTS = 4096;
constexpr uint32_t SITE_EMPTY = 0xFFFFFFFFu;

struct SiteSmem {
    uint32_t key[SITE_SLOTS];
    uint32_t cnt[SITE_SLOTS];
    unsigned long long bytes[SITE_SLOTS];
    unsigned long long ns[SITE_SLOTS];
};

__device__ __forceinline__ void site_add(SiteSmem& t, const A& a, uint32_t kind0, uint32_t site,
                                         uint64_t wb, uint64_t wn) {
    const uint32_t key = kind0 * ODP_MAX_SITES + site;
    uint32_t slot = (key * 2654435761u) >> (32 - 12);
    for (int probe = 0; probe < 32; ++probe) {
        const uint32_t old = atomicCAS(&t.key[slot], SITE_EMPTY, key);
        if (old == SITE_EMPTY || old == key) {
            atomicAdd(&t.cnt[slot], 1u);
            atomicAdd(&t.bytes[slot], (unsigned long long)wb);
            atomicAdd(&t.ns[slot], (unsigned long long)wn);
            return;
        }
        slot = (slot + 1) & (SITE_SLOTS - 1);
    }
    unsigned long long* row = a.sites + 3ull * key;
    atomicAdd(row + 0, 1ull);
    atomicAdd(row + 1, (unsigned long long)wb);
    atomicAdd(row + 2, (unsigned long long)wn);
}

// Persistent blocks; each warp walks 32-event chunks on its own: every
// finding is computed once, placed at (scanned chunk offset of its kind +
// rank in the chunk), added to the block's site table and the per-kind
// totals, and its wasted events are marked.  No block barrier inside the loop.
constexpr int EMW_THREADS = 512;

// Chunks ahead of the current one whose coalesced reads a warp prefetches
// into L2, so its first wait of a chunk is on L2 rather than DRAM.
constexpr uint32_t EMW_PREFETCH_AHEAD = 2;

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The 18 lines chunk cn reads before its first wait (its events' times,
// bytes, sites, deletes and partners) and its five scanned offsets, one line
// per lane; lines that start past the last event are skipped.
__device__ __forceinline__ void em_prefetch_chunk(const A& a, const uint32_t* wscan, uint32_t nch,
                                                  uint32_t cn, int lane) {
    if (cn >= nch || lane >= 18) return;
    const uint32_t base = cn * 32;
    uint32_t e = base;
    const void* p;
    if (lane < 4) e = base + 8 * lane, p = a.col.tt + e;
    else if (lane < 6) e = base + 16 * (lane - 4), p = a.col.bytes + e;
    else if (lane < 8) e = base + 16 * (lane - 6), p = a.drt + e;
    else if (lane == 8) p = a.col.site + base;
    else if (lane == 9) p = a.del_of + base;
    else if (lane == 10) p = a.ra + base;
    else if (lane == 11) p = a.ua + base;
    else if (lane == 12) p = a.ut + base;
    else p = wscan + (size_t)(lane - 13) * nch + cn;
    if (e < a.n) prefetch_l2(p);
}

// Sets event e's wasted bit; returns its duration if this call set it.
__device__ __forceinline__ uint64_t mark_wasted(const A& a, uint32_t e, uint64_t duration) {
    const uint32_t bit = 1u << (e & 31);
    return (atomicOr(a.wbits + (e >> 5), bit) & bit) ? 0 : duration;
}

__global__ void __launch_bounds__(EMW_THREADS) k_em_write(A a, const uint32_t* wscan, uint32_t nch) {
    pdl_entry();
    if (failed(a)) return;
    extern __shared__ __align__(16) unsigned char em_dyn[];
    SiteSmem& st = *reinterpret_cast<SiteSmem*>(em_dyn);
    __shared__ uint32_t chunk_off[EMW_THREADS / 32][5];  // the chunk's scanned offset per kind
    const int lane = threadIdx.x & 31;
    uint32_t* my_off = chunk_off[threadIdx.x >> 5];
    const uint32_t lt = (1u << lane) - 1;
    odp_finding* items = a.out.items;
    const uint64_t cap = a.out.capacity;
    for (int i = threadIdx.x; i < SITE_SLOTS; i += blockDim.x) {
        st.key[i] = SITE_EMPTY;
        st.cnt[i] = 0;
        st.bytes[i] = 0;
        st.ns[i] = 0;
    }
    __syncthreads();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long saved = 0;
    for (uint32_t k = 1; k < EMW_PREFETCH_AHEAD; ++k) em_prefetch_chunk(a, wscan, nch, gw + k * nw, lane);
    for (uint32_t c = gw; c < nch; c += nw) {
        const uint32_t i = c * 32 + lane;
        const bool valid = i < a.n;
        em_prefetch_chunk(a, wscan, nch, c + EMW_PREFETCH_AHEAD * nw, lane);
        // First loads: the partner arrays, and with them (before knowing whether
        // the event has a finding) its own record and the delete that closes
        // it, so a chunk waits for memory twice, not three times.
        uint32_t part[5];
        uint32_t bal[5];
        uint32_t any = 0;
        const uint32_t iv = valid ? i : 0u;
        const uint4 o0 = __ldg(a.col.tt + iv);  // t_start, t_end
        const uint64_t own_bytes = __ldg(reinterpret_cast<const unsigned long long*>(a.col.bytes) + iv);
        const uint32_t site = __ldg(a.col.site + iv);
        const uint32_t del = valid ? __ldg(a.del_of + i) : NONE32;
        const uint32_t off = lane < 5 ? __ldg(wscan + (size_t)lane * nch + c) : 0u;
        for (int kind = 0; kind < 5; ++kind) {
            part[kind] = valid ? partner_of(a, kind + 1, i) : NONE32;
            bal[kind] = __ballot_sync(ODP_FULL_MASK, part[kind] != NONE32);
            any |= bal[kind];
        }
        __syncwarp();  // the previous chunk's stores have read my_off
        if (lane < 5) my_off[lane] = off;
        __syncwarp();
        // Wasted events: the event itself for DD, RA, UA and UT findings (one
        // atomic per chunk), the partner for RT, the delete for RA and UA.
        // Whoever sets an event's bit adds its duration to the saved time, so
        // the union is summed once.
        const uint32_t own = bal[ODP_DD - 1] | bal[ODP_RA - 1] | bal[ODP_UA - 1] | bal[ODP_UT - 1];
        // (the old bits are read back only at the end of the chunk)
        uint32_t own_old = 0;
        if (lane == 0 && own) own_old = atomicOr(a.wbits + c, own);
        if (any & (1u << lane)) {
            const uint32_t d = part[ODP_RA - 1] != NONE32 ? del : NONE32;
            // Second loads: partner sites, the RT partner's times and bytes, the UA
            // partner's and the RA delete's times.
            uint32_t psite[5];
#pragma unroll
            for (int kind = 0; kind < 5; ++kind) {
                const uint32_t p = part[kind];
                psite[kind] = (p != NONE32 && p != NOPART) ? __ldg(a.col.site + p) : 0xFFFFFFFFu;
            }
            const uint32_t p_rt = part[ODP_RT - 1], p_ua = part[ODP_UA - 1];
            // (from the columns: their lines are shared with nearby events'
            // own reads, where whole records would each take a line of their own)
            const uint4 z4 = make_uint4(0, 0, 0, 0);
            const uint4 rt0 = p_rt != NONE32 ? __ldg(a.col.tt + p_rt) : z4;
            uint4 rt2 = z4;
            if (p_rt != NONE32) {
                const uint64_t by = __ldg(reinterpret_cast<const unsigned long long*>(a.col.bytes) + p_rt);
                rt2 = make_uint4((uint32_t)by, (uint32_t)(by >> 32), 0, 0);
            }
            const uint4 ua0 = (p_ua != NONE32 && p_ua != NOPART) ? __ldg(a.col.tt + p_ua) : z4;
            const uint4 d0 = d != NONE32 ? __ldg(a.col.tt + d) : z4;
            // Stores.
            const uint64_t t0 = lohi(o0.x, o0.y), t1 = lohi(o0.z, o0.w);
#pragma unroll
            for (int kind = 0; kind < 5; ++kind) {
                const uint32_t p = part[kind];
                if (p == NONE32) continue;
                const bool np = p == NOPART;
                uint64_t wb = own_bytes, wn = t1 - t0;
                switch (kind + 1) {
                    case ODP_RT:
                        wb = lohi(rt2.x, rt2.y);
                        wn = lohi(rt0.z, rt0.w) - lohi(rt0.x, rt0.y);
                        saved += mark_wasted(a, p, wn);
                        break;
                    case ODP_RA:
                        if (d != NONE32) {
                            const uint64_t dd = lohi(d0.z, d0.w) - lohi(d0.x, d0.y);
                            wn += dd;
                            saved += mark_wasted(a, d, dd);
                        }
                        break;
                    case ODP_UA:
                        if (!np) {
                            const uint64_t dp = lohi(ua0.z, ua0.w) - lohi(ua0.x, ua0.y);
                            wn += dp;
                            saved += mark_wasted(a, p, dp);
                        }
                        break;
                    default:  // DD, UT: the event itself (marked above)
                        break;
                }
                site_add(st, a, kind, site, wb, wn);
                const uint64_t pos = (uint64_t)my_off[kind] + __popc(bal[kind] & lt);
                if (pos < cap)
                    store_finding(items, pos, kind + 1, site, psite[kind], i,
                                  np ? ODP_NO_EVENT : (uint64_t)p, wb, wn);
            }
        }
        own_old = __shfl_sync(ODP_FULL_MASK, own_old, 0);
        if ((own >> lane) & 1 & ~(own_old >> lane)) saved += lohi(o0.z, o0.w) - lohi(o0.x, o0.y);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SITE_SLOTS; i += blockDim.x) {
        if (st.key[i] == SITE_EMPTY) continue;
        unsigned long long* row = a.sites + 3ull * st.key[i];
        atomicAdd(row + 0, (unsigned long long)st.cnt[i]);
        atomicAdd(row + 1, st.bytes[i]);
        atomicAdd(row + 2, st.ns[i]);
    }
    for (int d = 16; d > 0; d >>= 1) saved += __shfl_xor_sync(ODP_FULL_MASK, saved, d);
    if (lane == 0 && saved) atomicAdd(&a.h->saved_ns, saved);
}

// site rows: flags over the dense [kind][site] table (then compaction), and
// the per-kind totals of the summary as sums of the rows (every finding was
// added to exactly one row).  A warp's 32 rows share one kind.
__global__ void k_site_flags(A a, uint32_t* flags) {
    pdl_entry();
    const bool bad = failed(a);
    GRID_STRIDE(r, 5u * ODP_MAX_SITES) {
        const unsigned long long* row = a.sites + 3ull * r;
        unsigned long long c = bad ? 0 : row[0], wb = bad ? 0 : row[1], wn = bad ? 0 : row[2];
        flags[r] = c != 0;
        for (int d = 16; d > 0; d >>= 1) {
            c += __shfl_xor_sync(ODP_FULL_MASK, c, d);
            wb += __shfl_xor_sync(ODP_FULL_MASK, wb, d);
            wn += __shfl_xor_sync(ODP_FULL_MASK, wn, d);
        }
        if ((threadIdx.x & 31) == 0 && c) {
            const uint32_t kind = r / ODP_MAX_SITES + 1;
            atomicAdd(&a.h->count[kind], c);
            atomicAdd(&a.h->bytes[kind], wb);
            atomicAdd(&a.h->ns[kind], wn);
        }
    }
}

__global__ void k_site_write(A a, const uint32_t* flags, const uint32_t* pos) {
    pdl_entry();
    if (failed(a)) return;
    GRID_STRIDE(r, 5u * ODP_MAX_SITES) {
        if (!flags[r] || pos[r] >= a.out.sites_capacity) continue;
        odp_site_row row;
        row.site = r % ODP_MAX_SITES;
        row.kind = (uint8_t)(r / ODP_MAX_SITES + 1);
        row.pad[0] = row.pad[1] = row.pad[2] = 0;
        row.count = a.sites[3ull * r];
        row.wasted_bytes = a.sites[3ull * r + 1];
        row.wasted_ns = a.sites[3ull * r + 2];
        a.out.sites[pos[r]] = row;
    }
}

__global__ void k_finalize(A a, const uint32_t* n_findings, const uint32_t* n_rows) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    odp_summary* S = a.out.summary;
    const Hdr* h = a.h;
    if (h->err != NO_ERR || h->scan_fault) {
        uint64_t* z = (uint64_t*)S;
        for (size_t k = 0; k < sizeof(odp_summary) / 8; ++k) z[k] = 0;
        *a.out.count = 0;
        *a.out.sites_count = 0;
        *a.out.status = h->err != NO_ERR ? -(int32_t)(h->err & 0xFF) : ODP_ERR_TIMEOUT;
        return;
    }
    S->n_events = a.n;
    S->n_transfers = h->nX;
    S->n_allocs = h->n_allocs;
    S->n_deletes = h->n_deletes;
    S->n_kernels = h->nK;
    S->n_pairs = h->n_pairs;
    S->n_unpaired_allocs = h->n_allocs - h->n_pairs;
    S->n_unmatched_deletes = h->unmatched;
    for (int k = 0; k < 6; ++k) {
        S->count[k] = h->count[k];
        S->wasted_bytes[k] = h->bytes[k];
        S->wasted_ns[k] = h->ns[k];
    }
    const uint64_t begin = a.n ? a.ev.t0(0) : 0;
    const uint64_t end = h->t_end_max;
    S->trace_begin_ns = begin;
    S->trace_end_ns = end;
    S->trace_span_ns = end - begin;
    S->saved_ns = h->saved_ns;
    S->speedup_num = end - begin;
    S->speedup_den = (end - begin) > h->saved_ns ? (end - begin) - h->saved_ns : 0;
    const uint64_t total = *n_findings, rows = *n_rows;
    *a.out.count = total;
    *a.out.sites_count = rows;
    *a.out.status = (total > a.out.capacity || rows > a.out.sites_capacity) ? ODP_WARN_TRUNCATED : ODP_OK;
}

__global__ void k_empty_outputs(odp_findings out) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t* z = (uint64_t*)out.summary;
    for (size_t k = 0; k < sizeof(odp_summary) / 8; ++k) z[k] = 0;
    *out.count = 0;
    *out.sites_count = 0;
    *out.status = ODP_OK;
}

}  // namespace

// prim::table_clear for table type T (the overload picked by type).
template <class T>
void clear_table(const T& t, const uint32_t* count, uint32_t count_max, int grid, cudaStream_t s) {
    void (*kernel)(T, const uint32_t*, uint32_t) = prim::table_clear;
    pdl(kernel, grid, TPB, 0, s, t, count, count_max);
}

static int grid_for(uint64_t n, int sms) {
    uint64_t g = (n + TPB - 1) / TPB;
    uint64_t cap = (uint64_t)sms * 16;
    return (int)std::max<uint64_t>(1, std::min(g, cap));
}

static int an_run(const odp_event* events, uint64_t n64, const odp_findings* outp,
                  cudaStream_t s) {
    if (!outp) return ODP_ERR_INVALID_ARG;
    const odp_findings out = *outp;
    if (!out.count || !out.sites_count || !out.summary || !out.status) return ODP_ERR_INVALID_ARG;
    if (out.capacity > 0 && !out.items) return ODP_ERR_INVALID_ARG;
    if (((uintptr_t)out.items & 15) != 0) return ODP_ERR_INVALID_ARG;  // 16-byte stores
    if (out.sites_capacity > 0 && !out.sites) return ODP_ERR_INVALID_ARG;
    if (n64 > 0 && !events) return ODP_ERR_INVALID_ARG;
    if (((uintptr_t)events & 15) != 0) return ODP_ERR_INVALID_ARG;  // records are read as 16-byte words
    if (n64 >= 0xFFFFFFF0ull) return ODP_ERR_UNSUPPORTED;
    if (n64 == 0) {
        pdl(k_empty_outputs, 1, 1, 0, s, out);
        return cuda_status(cudaGetLastError());
    }
    const uint32_t n = (uint32_t)n64;
    const int sms = device_sm_count();
    int st = ODP_OK;

    uint32_t cap_max = 1024;
    while (cap_max < (uint64_t)n + n / 4) cap_max <<= 1;

    // ---- scratch layout
    size_t bytes = 0;
    auto carve = [&](size_t sz) {
        size_t o = bytes;
        bytes = align_up(bytes + std::max<size_t>(sz, 16), 256);
        return o;
    };
    const size_t N4 = 4ull * (n + 2);
    const size_t o_h = carve(sizeof(Hdr));
    const size_t o_cls = carve(N4);
    const uint32_t nch = (n + 31) / 32;
    const size_t o_wcnt = carve(4ull * (5ull * nch + 2));
    const size_t o_wscan = carve(4ull * (5ull * nch + 2));
    const size_t o_X = carve(N4), o_P = carve(N4), o_K = carve(N4), o_U = carve(N4);
    const size_t PS = (n + 2 + 3) & ~size_t(3);  // partner array stride: 16-byte aligned rows
    const size_t o_part = carve(6 * 4 * PS);  // dd rt ra ua ut del_of
    const size_t o_wasted = carve(4ull * ((n + 31) / 32) + 16);
    const size_t o_bad = carve(n + 16);
    const size_t o_slot = carve(N4), o_sk = carve(N4), o_sv = carve(N4), o_k2 = carve(N4),
                 o_v2 = carve(N4), o_f1 = carve(N4), o_f2 = carve(N4), o_id1 = carve(N4),
                 o_id2 = carve(N4), o_H = carve(N4), o_R = carve(N4), o_stk = carve(N4),
                 o_pq = carve(N4);
    const size_t o_uc = carve(n + 16);
    const size_t o_ctt = carve(16ull * n), o_chd = carve(16ull * n), o_cby = carve(8ull * n),
                 o_cfp = carve(16ull * n), o_cst = carve(4ull * n);
    const size_t o_kse = carve(16ull * (n + 2));  // ks | ke (also 16 B per endpoint segment)
    const size_t o_dev = carve(2 * 4 * NDEV);
    const size_t o_sites = carve(8ull * 3 * 5 * ODP_MAX_SITES);
    const size_t o_sflag = carve(4ull * 5 * ODP_MAX_SITES), o_spos = carve(4ull * 5 * ODP_MAX_SITES);
    const size_t o_misc = carve(64);
    const size_t o_keys_alt = carve(N4), o_vals_alt = carve(N4);
    const size_t o_hist = carve(4 * prim::sort_hist_words(n));
    const size_t scan_words = std::max(prim::scan_tmp_words(256u * ((n + prim::SORT_TILE - 1) / prim::SORT_TILE + 1)),
                                       std::max(prim::scan_tmp_words(n), prim::scan_tmp_words(5 * ODP_MAX_SITES)));
    const size_t o_scan = carve(4 * (scan_words + 16));
    const size_t o_tslots = carve(sizeof(prim::Slot) * ((size_t)cap_max + 1));

    uint8_t* b = (uint8_t*)scratch_get(SLOT_AN_MAIN, bytes, s, &st);
    if (!b) return st;

    A a;
    a.ev.p = (const uint8_t*)events;
    a.n = n;
    a.h = (Hdr*)(b + o_h);
    a.cls = (uint32_t*)(b + o_cls);
    a.X = (uint32_t*)(b + o_X);
    a.P = (uint32_t*)(b + o_P);
    a.K = (uint32_t*)(b + o_K);
    a.U = (uint32_t*)(b + o_U);
    uint32_t* part = (uint32_t*)(b + o_part);
    a.drt = reinterpret_cast<uint2*>(part);  // two rows
    a.ra = part + 2 * PS;
    a.ua = part + 3 * PS;
    a.ut = part + 4 * PS;
    a.del_of = part + 5 * PS;
    a.wbits = (uint32_t*)(b + o_wasted);
    a.bad = b + o_bad;
    a.slot = (uint32_t*)(b + o_slot);
    a.sk = (uint32_t*)(b + o_sk);
    a.sv = (uint32_t*)(b + o_sv);
    a.k2 = (uint32_t*)(b + o_k2);
    a.v2 = (uint32_t*)(b + o_v2);
    a.f1 = (uint32_t*)(b + o_f1);
    a.f2 = (uint32_t*)(b + o_f2);
    a.id1 = (uint32_t*)(b + o_id1);
    a.id2 = (uint32_t*)(b + o_id2);
    a.H = (uint32_t*)(b + o_H);
    a.R = (uint32_t*)(b + o_R);
    a.stk = (uint32_t*)(b + o_stk);
    a.pq = (uint32_t*)(b + o_pq);
    a.uc = b + o_uc;
    a.col.tt = (uint4*)(b + o_ctt);
    a.col.hd = (uint4*)(b + o_chd);
    a.col.bytes = (uint64_t*)(b + o_cby);
    a.col.fp = (uint4*)(b + o_cfp);
    a.col.site = (uint32_t*)(b + o_cst);
    a.ks = (uint64_t*)(b + o_kse);
    a.ke = a.ks + (n + 2);
    a.dstart = (uint32_t*)(b + o_dev);
    a.dend = a.dstart + NDEV;
    a.sites = (unsigned long long*)(b + o_sites);
    uint32_t* sflag = (uint32_t*)(b + o_sflag);
    uint32_t* spos = (uint32_t*)(b + o_spos);
    uint32_t* misc = (uint32_t*)(b + o_misc);  // [0] total findings, [1] site rows, [2] scan total, [3] sort histogram length
    a.tab.keys = (Key128*)(b + o_tslots);
    a.tab.vals = (uint32_t*)(b + o_tslots + sizeof(Key128) * ((size_t)cap_max + 1));
    a.tab.cap_max = cap_max;
    a.tab.cap_dev = &a.h->tcap;
    a.ktab.keys = (Key128*)(b + o_tslots);
    a.ktab.cap_max = cap_max;
    a.ktab.cap_dev = &a.h->tcap;
    a.gid = a.tab.vals;
    a.out = out;
    prim::SortTmp srt;
    srt.keys_alt = (uint32_t*)(b + o_keys_alt);
    srt.vals_alt = (uint32_t*)(b + o_vals_alt);
    srt.hist = (uint32_t*)(b + o_hist);
    srt.scan_tmp = (uint32_t*)(b + o_scan);
    srt.hlen = misc + 3;
    srt.fault = &a.h->scan_fault;
    srt.pdl = true;  // the whole chain uses programmatic dependent launch
    uint32_t* scan_tmp = srt.scan_tmp;

    const int bits_n = prim::bit_length(n);              // keys < n + 1
    const int bits_slot = prim::bit_length(cap_max + 1);  // slot keys <= cap_max + 1
    a.pack_alloc = bits_slot <= 31;
    const int gX = grid_for(n, sms);
    const int clear_grid = sms * 8;

    // ---- init
    ODP_CHECK_CUDA(cudaMemsetAsync(a.h, 0, sizeof(Hdr), s));
    ODP_CHECK_CUDA(cudaMemsetAsync(&a.h->err, 0xFF, 8, s));
    ODP_CHECK_CUDA(cudaMemsetAsync(part, 0xFF, 6 * 4 * PS, s));
    ODP_CHECK_CUDA(cudaMemsetAsync(a.wbits, 0, 4ull * ((n + 31) / 32) + 16, s));
    ODP_CHECK_CUDA(cudaMemsetAsync(a.dstart, 0, 2 * 4 * NDEV, s));
    ODP_CHECK_CUDA(cudaMemsetAsync(a.sites, 0, 8ull * 3 * 5 * ODP_MAX_SITES, s));
    ODP_CHECK_CUDA(cudaMemsetAsync(scan_tmp, 0, 4 * (scan_words + 16), s));
    // the all-ones fingerprint's group key (its first event, an atomic minimum)
    ODP_CHECK_CUDA(cudaMemsetAsync(a.gid + cap_max, 0xFF, 4, s));

    // ---- validate, lists
    uint32_t* ccnt = (uint32_t*)(b + o_wcnt);
    uint32_t* cscan = (uint32_t*)(b + o_wscan);
    pdl(k_validate, sms * 16, TPB, 0, s, a, ccnt, nch);
    prim::exclusive_scan(ccnt, cscan, nullptr, 4 * nch, misc + 2, scan_tmp, s, srt.fault, true);
    pdl(k_list_lengths, 1, 32, 0, s, a, cscan, misc + 2, nch);
    pdl(k_compact, sms * 16, TPB, 0, s, a, cscan, nch);
    uint32_t* nX = &a.h->nX;
    uint32_t* nP = &a.h->nP;
    uint32_t* nK = &a.h->nK;
    uint32_t* nU = &a.h->nU;

    // ---- Alg. 1: content ids, first receivers
    clear_table(a.ktab, nX, n, clear_grid, s);
    pdl(k_x_insert_fp, gX, TPB, 0, s, a);
    pdl(k_x_cid, gX, TPB, 0, s, a);

    // ---- Alg. 2
    prim::radix_sort(a.sk, a.sv, nX, n, bits_n, srt, s);
    pdl(k_rt_flags, gX, TPB, 0, s, a);
    prim::exclusive_scan(a.f1, a.id1, nX, n, &a.h->nseg, scan_tmp, s, srt.fault, true);
    prim::exclusive_scan(a.f2, a.id2, nX, n, &a.h->nrun, scan_tmp, s, srt.fault, true);
    pdl(k_rt_starts, gX, TPB, 0, s, a);
    pdl(k_rt_check, gX, TPB, 0, s, a);
    pdl(k_rt_partner, gX, TPB, 0, s, a);
    // groups with more than two endpoints
    uint32_t* nB = &a.h->nB;
    pdl(k_mx_flag, gX, TPB, 0, s, a);
    prim::exclusive_scan(a.f2, a.id2, &a.h->mx_n, n, nB, scan_tmp, s, srt.fault, true);
    pdl(k_mx_scatter, gX, TPB, 0, s, a);
    prim::radix_sort(a.k2, a.v2, nB, n, 8, srt, s);
    pdl(k_mx_gkey, gX, TPB, 0, s, a);
    prim::radix_sort(a.k2, a.v2, nB, n, bits_n, srt, s);
    pdl(k_mx_heads, gX, TPB, 0, s, a);
    prim::exclusive_scan(a.f2, a.id2, nB, n, &a.h->nsegB, scan_tmp, s, srt.fault, true);
    pdl(k_mx_starts, gX, TPB, 0, s, a);
    pdl(k_mx_late, gX, TPB, 0, s, a);
    pdl(k_mx_ok, gX, TPB, 0, s, a);
    pdl(k_mx_succ, gX, TPB, 0, s, a);
    prim::exclusive_scan(a.k2, a.sk, nB, n, nullptr, scan_tmp, s, srt.fault, true);
    pdl(k_mx_partner, gX, TPB, 0, s, a);

    // ---- pairs
    clear_table(a.ktab, nP, n, clear_grid, s);
    pdl(k_p_insert, gX, TPB, 0, s, a);
    pdl(k_gid_keys, gX, TPB, 0, s, a, a.sk, nP, a.pack_alloc ? 0x80000000u : 0u);
    prim::radix_sort(a.sk, a.sv, nP, n, bits_slot, srt, s, &a.h->n_gid_p);
    pdl(k_seg_heads, gX, TPB, 0, s, a, nP);
    prim::exclusive_scan(a.f1, a.id1, nP, n, &a.h->nseg2, scan_tmp, s, srt.fault, true);
    pdl(k_seg_starts, gX, TPB, 0, s, a, nP, &a.h->nseg2);
    pdl(k_p_check, gX, TPB, 0, s, a);
    pdl(k_p_match, gX, TPB, 0, s, a);
    pdl(k_p_literal, gX, TPB, 0, s, a);

    // ---- Alg. 3
    clear_table(a.tab, &a.h->nA, n, clear_grid, s);
    pdl(k_ra_insert, gX, TPB, 0, s, a);
    pdl(k_ra_flag, gX, TPB, 0, s, a);

    // ---- kernels per device
    pdl(k_dev_keys, gX, TPB, 0, s, a, a.K, nK, &a.h->k_mixed);
    pdl(k_sort_count, 1, 32, 0, s, nK, &a.h->k_mixed, &a.h->k_sortn);
    prim::radix_sort(a.sk, a.sv, &a.h->k_sortn, n, 8, srt, s);
    pdl(k_k_bounds, gX, TPB, 0, s, a);
    pdl(k_k_pmax, NDEV, PMAX_THREADS, 0, s, a);

    // ---- Alg. 4
    pdl(k_ua, gX, TPB, 0, s, a);

    // ---- Alg. 5
    pdl(k_dev_keys, gX, TPB, 0, s, a, a.U, nU, &a.h->u_mixed);
    pdl(k_sort_count, 1, 32, 0, s, nU, &a.h->u_mixed, &a.h->u_sortn);
    prim::radix_sort(a.sk, a.sv, &a.h->u_sortn, n, 8, srt, s);
    pdl(k_ut_class, gX, TPB, 0, s, a);
    pdl(k_ut_heads, gX, TPB, 0, s, a);
    prim::exclusive_scan(a.f1, a.id1, nU, n, &a.h->nsegU, scan_tmp, s, srt.fault, true);
    clear_table(a.ktab, nU, n, clear_grid, s);
    pdl(k_ut_insert, gX, TPB, 0, s, a);
    pdl(k_gid_keys, gX, TPB, 0, s, a, a.k2, nU, 0u);
    prim::radix_sort(a.k2, a.v2, nU, n, bits_slot, srt, s, &a.h->n_gid_u);
    pdl(k_ut_next, gX, TPB, 0, s, a);

    // ---- emission
    uint32_t* wcnt = (uint32_t*)(b + o_wcnt);
    uint32_t* wscan = (uint32_t*)(b + o_wscan);
    pdl(k_em_count, sms * 8, 256, 0, s, a, wcnt, nch);
    prim::exclusive_scan(wcnt, wscan, nullptr, 5 * nch, misc + 0, scan_tmp, s, srt.fault, true);
    static std::atomic<bool> em_attr[256] = {};
    const int dev = current_device();
    if (dev < 256 && !em_attr[dev].load(std::memory_order_acquire)) {
        ODP_CHECK_CUDA(cudaFuncSetAttribute(k_em_write, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(SiteSmem)));
        em_attr[dev].store(true, std::memory_order_release);
    }
    pdl(k_em_write, sms * 2, EMW_THREADS, sizeof(SiteSmem), s, a, wscan, nch);
    pdl(k_site_flags, grid_for(5u * ODP_MAX_SITES, sms), TPB, 0, s, a, sflag);
    prim::exclusive_scan(sflag, spos, nullptr, 5u * ODP_MAX_SITES, misc + 1, scan_tmp, s, srt.fault,
                         true);
    pdl(k_site_write, grid_for(5u * ODP_MAX_SITES, sms), TPB, 0, s, a, sflag, spos);
    pdl(k_finalize, 1, 32, 0, s, a, misc + 0, misc + 1);
    return cuda_status(cudaGetLastError());
}

}  // namespace odp

extern "C" int odp_analyze(const odp_event* events, uint64_t n, const odp_findings* out,
                           cudaStream_t stream) {
    return odp::an_run(events, n, out, stream);
}
