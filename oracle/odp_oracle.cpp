// odp_oracle.cpp -- CPU oracle for the data-mapping analysis hot path.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
// reference that the GPU library is checked against.  Only the test suite,
// the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
// no code, header, table or constant generator with the CUDA library: every
// structure and constant below is declared or derived here on its own.
//
// Contents
//   1. FP128 v1, the project's 128-bit chunked tree hash, computed byte-wise
//      (the paper, Sec. 5.1, stores a hash of every transferred buffer and
//      assumes it is collision-free; the hash itself is project-defined).
//   2. Algorithms 1-5 of the paper (Sec. 5), transcribed step by step with
//      std::map / std::deque, plus the readings the paper leaves open:
//        - GetAllocDeletePairs (used by Alg. 3 and 4, never defined): a DELETE
//          closes the nearest preceding unpaired ALLOC with the same
//          (device, device address); allocations never deleted are not pairs.
//        - Alg. 3 appends <alloc_event, event>: read `event` as the delete.
//        - Alg. 1/2 operate on transfers only (to-device, from-device,
//          device-to-device); Alg. 5 on to-device transfers only.
//        - Host device number is -1.
//   3. The optimisation-potential estimate of Sec. 7.6 (total time minus the
//      time of eliminable transfers/allocations), per finding and as a
//      union over flagged events.
//
// Parity status: FP128 is project-defined, so it is pinned by the published
// SplitMix64 test vectors (its constants), by algebraic invariants (every
// single 16-byte word change alters the hash, the mixers are bijections with
// explicit inverses), by running each lane backwards to its start constants
// (chain step and Feistel finish inverted by the tests), by the closed form
// of the lane tree (lane l reaches the root through G^popcount(l)), by the
// leaf constants recovered through the inverse of Q, by worked examples
// checked step by step, by tree-shape equivalence and by collision tests; the
// analysis is pinned by the paper's worked listings, Table 2 count semantics
// and brute-force definitions on exhaustive small traces.  The predicted-
// speedup *accuracy* against real applications is parity unpinned (it needs
// the paper's applications).
//
// Build: g++ -O2 -shared -fPIC -o liboracle.so odp_oracle.cpp

#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <map>
#include <deque>
#include <vector>
#include <tuple>
#include <algorithm>
#include <utility>

namespace {

// ---------------------------------------------------------------------------
// 1. FP128 v1
// ---------------------------------------------------------------------------

typedef uint64_t u64;
typedef uint32_t u32;

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the state advances by the
// golden-ratio increment and each output is the state passed through the
// published finaliser.  Output i (0-based) of a generator seeded with s.
u64 splitmix64_output(u64 seed, u64 i) {
    u64 z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// All FP128 v1 constants are SplitMix64 outputs from this seed: the ASCII
// bytes "FP128_v1" read as a big-endian integer.
const u64 FP_SEED = 0x46503132385F7631ULL;

struct FpConstants {
    u64 c[96];
    FpConstants() {
        for (int i = 0; i < 96; ++i) c[i] = splitmix64_output(FP_SEED, (u64)i);
    }
    u64 odd(int i) const { return c[i] | 1ULL; }
};

const FpConstants& K() {
    static FpConstants k;
    return k;
}

struct U128 {
    u64 x, y;  // x = low half, y = high half
};

// Per-word chain step: multiply by an odd constant, fold the high 32 bits
// down, multiply by a second odd constant.  Each of the three steps is a
// bijection of the 64-bit state, so the step is one too.
u64 chain_step(u64 v, u64 k1, u64 k2) {
    u64 t = v * k1;
    t = t ^ (t >> 32);
    t = t * k2;
    return t;
}

// The 128-bit mixer used for leaves (Q), tree nodes (P) and the final output
// (Z); each one uses its own four odd multipliers.  Every step is invertible:
// odd multiplications and xors of one half with a function of the other.
U128 mix128(U128 s, u64 k0, u64 k1, u64 k2, u64 k3) {
    u64 x = s.x, y = s.y;
    x = x * k0;
    y = y ^ (x >> 29);
    y = y * k1;
    x = x ^ (y >> 32);
    x = x * k2;
    y = y ^ (x >> 32);
    y = y * k3;
    x = x ^ (y >> 29);
    U128 r = {x, y};
    return r;
}

U128 mix_Q(U128 s) { return mix128(s, K().odd(6), K().odd(7), K().odd(8), K().odd(9)); }
U128 mix_P(U128 s) { return mix128(s, K().odd(10), K().odd(11), K().odd(12), K().odd(13)); }
U128 mix_Z(U128 s) { return mix128(s, K().odd(14), K().odd(15), K().odd(16), K().odd(17)); }

// G(x, y) = (y, x ^ y): the linear map applied to the right operand of every
// combine; G and I ^ G are both invertible.
U128 G(U128 s) {
    U128 r = {s.y, s.x ^ s.y};
    return r;
}

U128 xor128(U128 a, U128 b) {
    U128 r = {a.x ^ b.x, a.y ^ b.y};
    return r;
}

// Little-endian u64 from 8 bytes.
u64 load_le64(const uint8_t* p) {
    u64 v = 0;
    for (int i = 7; i >= 0; --i) v = (v << 8) | (u64)p[i];
    return v;
}

const u64 CHUNK = 4096;

// State of lane l (0..31) of a chunk zero-padded to 4096 bytes: the lane
// absorbs words l, l+32, ..., l+224 into two chains, then a two-round
// Feistel couples the two chains.
U128 lane_state(const uint8_t* padded, int l) {
    u64 a = K().c[32 + 2 * l];
    u64 b = K().c[33 + 2 * l];
    for (int j = 0; j < 8; ++j) {
        int w = l + 32 * j;
        u64 lo = load_le64(padded + 16 * w);
        u64 hi = load_le64(padded + 16 * w + 8);
        a = chain_step(a ^ lo, K().odd(0), K().odd(1));
        b = chain_step(b ^ hi, K().odd(2), K().odd(3));
    }
    a = a ^ (b * K().odd(4));
    b = b ^ (a * K().odd(5));
    U128 s = {a, b};
    return s;
}

// The chunk at `p` with `r` valid bytes, zero-padded to 4096 bytes.
void pad_chunk(const uint8_t* p, u64 r, uint8_t* padded) {
    std::memset(padded, 0, (size_t)CHUNK);
    std::memcpy(padded, p, (size_t)r);
}

// Leaf of one chunk: `r` valid bytes (1..4096) starting at `p`.
U128 chunk_leaf(const uint8_t* p, u64 r) {
    // The chunk zero-padded to 4096 bytes, as 256 sixteen-byte words.
    uint8_t padded[CHUNK];
    pad_chunk(p, r, padded);

    U128 lane[32];
    for (int l = 0; l < 32; ++l) lane[l] = lane_state(padded, l);

    // Lane combine: a complete binary tree over the 32 lanes, left operand is
    // the lower lane range; node = left ^ G(right).
    for (int width = 1; width < 32; width *= 2) {
        for (int l = 0; l + width < 32; l += 2 * width) {
            lane[l] = xor128(lane[l], G(lane[l + width]));
        }
    }
    U128 root = lane[0];

    // Leaf finalisation mixes in the valid byte count and the leaf domain.
    U128 t = {root.x ^ r ^ K().c[18], root.y ^ K().c[19]};
    return mix_Q(t);
}

// Interior node over a left and right subtree covering `count` leaves.
U128 tree_node(U128 left, U128 right, u64 count) {
    U128 g = G(right);
    U128 t = {left.x ^ g.x ^ count, left.y ^ g.y ^ K().c[20]};
    return mix_P(t);
}

// Left-balanced binary tree over leaves[lo, hi): split at the largest power
// of two strictly below the leaf count (the shape of RFC 6962 Merkle trees).
U128 tree_root(const std::vector<U128>& leaves, u64 lo, u64 hi) {
    u64 n = hi - lo;
    if (n == 1) return leaves[(size_t)lo];
    u64 k = 1;
    while (k * 2 < n) k *= 2;
    U128 left = tree_root(leaves, lo, lo + k);
    U128 right = tree_root(leaves, lo + k, hi);
    return tree_node(left, right, n);
}

U128 fp128(const uint8_t* data, u64 len) {
    u64 n_chunks = (len + CHUNK - 1) / CHUNK;
    U128 root;
    if (len == 0) {
        root.x = K().c[22];
        root.y = K().c[23];
    } else {
        std::vector<U128> leaves;
        for (u64 c = 0; c < n_chunks; ++c) {
            u64 off = c * CHUNK;
            u64 r = std::min(CHUNK, len - off);
            leaves.push_back(chunk_leaf(data + off, r));
        }
        root = tree_root(leaves, 0, n_chunks);
    }
    U128 t = {root.x ^ len, root.y ^ n_chunks ^ K().c[21]};
    return mix_Z(t);
}

// ---------------------------------------------------------------------------
// 2. Event log and findings (the oracle's own declarations of the 64-byte
//    event record and the 48-byte finding record).
// ---------------------------------------------------------------------------

#pragma pack(push, 1)
struct Event {
    u64 t_start_ns;
    u64 t_end_ns;
    u64 host_addr;
    u64 dev_addr;
    u64 bytes;
    u64 fp_lo;
    u64 fp_hi;
    u32 site_id;
    uint8_t kind;
    int8_t src_dev;
    int8_t dst_dev;
    uint8_t flags;
};
struct Finding {
    uint8_t kind;
    uint8_t pad0[3];
    u32 site;
    u32 partner_site;
    u32 pad1;
    u64 event;
    u64 partner;
    u64 wasted_bytes;
    u64 wasted_ns;
};
struct SiteRow {
    u32 site;
    uint8_t kind;
    uint8_t pad[3];
    u64 count;
    u64 wasted_bytes;
    u64 wasted_ns;
};
struct Summary {
    u64 n_events;
    u64 n_transfers;
    u64 n_allocs;
    u64 n_deletes;
    u64 n_kernels;
    u64 n_pairs;
    u64 n_unpaired_allocs;
    u64 n_unmatched_deletes;
    u64 count[6];         // indexed by finding kind 1..5
    u64 wasted_bytes[6];
    u64 wasted_ns[6];
    u64 trace_begin_ns;
    u64 trace_end_ns;
    u64 trace_span_ns;
    u64 saved_ns;         // union over flagged wasted events
    u64 speedup_num;      // predicted speedup = num / den (den 0: unbounded)
    u64 speedup_den;
};
#pragma pack(pop)

static_assert(sizeof(Event) == 64, "event record is 64 bytes");
static_assert(sizeof(Finding) == 48, "finding record is 48 bytes");
static_assert(sizeof(SiteRow) == 32, "site row is 32 bytes");

enum {
    K_ALLOC = 1, K_TO_DEV = 2, K_FROM_DEV = 3, K_DEV_TO_DEV = 4, K_DELETE = 5, K_KERNEL = 6
};
enum { F_DD = 1, F_RT = 2, F_RA = 3, F_UA = 4, F_UT = 5 };
enum {
    S_OK = 0, S_WARN_TRUNCATED = 1, S_ERR_INVALID_ARG = -1, S_ERR_MALFORMED = -5, S_ERR_UNSORTED = -6
};

const u64 NONE = ~0ULL;
const u32 MAX_SITES = 65536;
const u64 MAX_BYTES = 1ULL << 56;

bool is_transfer(const Event& e) {
    return e.kind == K_TO_DEV || e.kind == K_FROM_DEV || e.kind == K_DEV_TO_DEV;
}

u64 duration(const Event& e) { return e.t_end_ns - e.t_start_ns; }

// Record-level checks; returns true when the record is well formed.
bool record_ok(const Event& e) {
    if (e.t_end_ns < e.t_start_ns) return false;
    if (e.site_id >= MAX_SITES) return false;
    if (e.bytes >= MAX_BYTES) return false;
    switch (e.kind) {
        case K_TO_DEV:
            return e.bytes > 0 && e.src_dev == -1 && e.dst_dev >= 0;
        case K_FROM_DEV:
            return e.bytes > 0 && e.src_dev >= 0 && e.dst_dev == -1;
        case K_DEV_TO_DEV:
            return e.bytes > 0 && e.src_dev >= 0 && e.dst_dev >= 0 && e.src_dev != e.dst_dev;
        case K_ALLOC:
        case K_DELETE:
        case K_KERNEL:
            return e.dst_dev >= 0;
        default:
            return false;
    }
}

// Content identity used by the pattern algorithms: the fingerprint, or, in
// brute-force mode, an id shared by events whose payloads compare equal.
struct Content {
    u64 a, b;
    bool operator<(const Content& o) const { return a != o.a ? a < o.a : b < o.b; }
    bool operator==(const Content& o) const { return a == o.a && b == o.b; }
};

struct Out {
    std::vector<Finding> findings;
};

Finding make_finding(const std::vector<Event>& ev, int kind, u64 event, u64 partner,
                     u64 wasted_bytes, u64 wasted_ns) {
    Finding f;
    std::memset(&f, 0, sizeof f);
    f.kind = (uint8_t)kind;
    f.site = ev[(size_t)event].site_id;
    f.partner_site = partner == NONE ? 0xFFFFFFFFu : ev[(size_t)partner].site_id;
    f.event = event;
    f.partner = partner;
    f.wasted_bytes = wasted_bytes;
    f.wasted_ns = wasted_ns;
    return f;
}

// Algorithm 1, FindDuplicateTransfers.  Groups transfers by <hash, dest> and
// keeps the groups with two or more events.  Each event after the first of a
// group is one finding whose partner is the first event of the group.
void find_duplicate_transfers(const std::vector<Event>& ev, const std::vector<Content>& content,
                              const std::vector<u64>& data_op_events, Out& out) {
    std::vector<std::vector<u64>> duplicate_transfers;
    std::map<std::pair<Content, int>, std::vector<u64>> received;
    for (u64 idx : data_op_events) {
        std::pair<Content, int> key(content[(size_t)idx], ev[(size_t)idx].dst_dev);
        received[key].push_back(idx);
    }
    for (auto& kv : received) {
        if (kv.second.size() < 2) continue;
        duplicate_transfers.push_back(kv.second);
    }
    for (auto& group : duplicate_transfers) {
        u64 first = group[0];
        for (size_t i = 1; i < group.size(); ++i) {
            const Event& e = ev[(size_t)group[i]];
            out.findings.push_back(make_finding(ev, F_DD, group[i], first, e.bytes, duration(e)));
        }
    }
}

// Algorithm 2, FindRoundTrips, kept literal: peek does not dequeue, and the
// dequeue removes the front of received[<hash, tx.dest>].  One finding per
// <tx, rx> pair; the wasted transfer is the return trip rx.
void find_round_trips(const std::vector<Event>& ev, const std::vector<Content>& content,
                      const std::vector<u64>& data_op_events, Out& out) {
    std::map<std::tuple<Content, int, int>, std::vector<std::pair<u64, u64>>> round_trips;
    std::map<std::pair<Content, int>, std::deque<u64>> received;
    for (u64 idx : data_op_events) {
        std::pair<Content, int> key(content[(size_t)idx], ev[(size_t)idx].dst_dev);
        received[key].push_back(idx);
    }
    std::vector<std::pair<u64, u64>> pairs_in_order;
    for (u64 tx : data_op_events) {
        const Event& t = ev[(size_t)tx];
        std::pair<Content, int> rx_key(content[(size_t)tx], t.src_dev);
        auto it = received.find(rx_key);
        if (it == received.end() || it->second.empty()) {
            continue;  // not a round trip: the data is never sent back
        }
        std::tuple<Content, int, int> trip_key(content[(size_t)tx], t.src_dev, t.dst_dev);
        u64 rx = it->second.front();  // peek
        round_trips[trip_key].push_back(std::make_pair(tx, rx));
        pairs_in_order.push_back(std::make_pair(tx, rx));
        std::pair<Content, int> tx_key(content[(size_t)tx], t.dst_dev);
        received[tx_key].pop_front();  // never empty: tx itself was enqueued there
    }
    for (auto& pr : pairs_in_order) {
        const Event& rx = ev[(size_t)pr.second];
        out.findings.push_back(make_finding(ev, F_RT, pr.first, pr.second, rx.bytes, duration(rx)));
    }
}

struct AllocPair {
    u64 alloc;
    u64 del;  // NONE for an allocation that is never deleted
};

// GetAllocDeletePairs (reading): scan in chronological order; an ALLOC opens
// an entry for its (device, device address); a DELETE closes the most recent
// open entry for the same key.  Returns completed pairs ordered by the alloc
// index, the allocations never deleted, and the number of unmatched deletes.
void get_alloc_delete_pairs(const std::vector<Event>& ev, std::vector<AllocPair>& pairs,
                            std::vector<u64>& unpaired_allocs, u64& unmatched_deletes) {
    std::map<std::pair<int, u64>, std::vector<u64>> open;
    unmatched_deletes = 0;
    for (u64 i = 0; i < ev.size(); ++i) {
        const Event& e = ev[(size_t)i];
        std::pair<int, u64> key(e.dst_dev, e.dev_addr);
        if (e.kind == K_ALLOC) {
            open[key].push_back(i);
        } else if (e.kind == K_DELETE) {
            auto it = open.find(key);
            if (it == open.end() || it->second.empty()) {
                unmatched_deletes++;
                continue;
            }
            AllocPair p = {it->second.back(), i};
            it->second.pop_back();
            pairs.push_back(p);
        }
    }
    for (auto& kv : open)
        for (u64 a : kv.second) unpaired_allocs.push_back(a);
    std::sort(pairs.begin(), pairs.end(),
              [](const AllocPair& l, const AllocPair& r) { return l.alloc < r.alloc; });
    std::sort(unpaired_allocs.begin(), unpaired_allocs.end());
}

// Algorithm 3, FindRepeatedAllocs.  Pairs keyed by <host address, target
// device, bytes>; keys with two or more pairs are repeated allocations.  Each
// pair after the first is one finding, partner = the first pair's alloc.
void find_repeated_allocs(const std::vector<Event>& ev, const std::vector<AllocPair>& allocs,
                          Out& out) {
    std::map<std::tuple<u64, int, u64>, std::vector<AllocPair>> repeated_allocs;
    for (const AllocPair& p : allocs) {
        const Event& a = ev[(size_t)p.alloc];
        std::tuple<u64, int, u64> key(a.host_addr, a.dst_dev, a.bytes);
        repeated_allocs[key].push_back(p);
    }
    for (auto it = repeated_allocs.begin(); it != repeated_allocs.end();) {
        if (it->second.size() < 2)
            it = repeated_allocs.erase(it);
        else
            ++it;
    }
    for (auto& kv : repeated_allocs) {
        u64 first = kv.second[0].alloc;
        for (size_t i = 1; i < kv.second.size(); ++i) {
            const Event& a = ev[(size_t)kv.second[i].alloc];
            const Event& d = ev[(size_t)kv.second[i].del];
            out.findings.push_back(make_finding(ev, F_RA, kv.second[i].alloc, first, a.bytes,
                                                duration(a) + duration(d)));
        }
    }
}

// SortByDevice: events of each device, keeping chronological order.
std::map<int, std::vector<u64>> sort_by_device(const std::vector<Event>& ev,
                                               const std::vector<u64>& idx) {
    std::map<int, std::vector<u64>> by_dev;
    for (u64 i : idx) by_dev[ev[(size_t)i].dst_dev].push_back(i);
    return by_dev;
}

// Algorithm 4, FindUnusedAllocs.  Per device, a monotone pointer walks the
// kernels while their end precedes the allocation's start; the allocation is
// unused when the pointer ran off the end or the kernel it stops at starts
// after the delete ends.  Allocations that are never deleted take the trace
// end as their delete end (and have no partner).
void find_unused_allocs(const std::vector<Event>& ev, const std::vector<u64>& tgt_events,
                        const std::vector<AllocPair>& pairs, const std::vector<u64>& unpaired,
                        u64 trace_end, Out& out) {
    std::vector<AllocPair> alloc_events(pairs);
    for (u64 a : unpaired) {
        AllocPair p = {a, NONE};
        alloc_events.push_back(p);
    }
    std::sort(alloc_events.begin(), alloc_events.end(),
              [](const AllocPair& l, const AllocPair& r) { return l.alloc < r.alloc; });

    std::map<int, std::vector<u64>> device_tgt_events = sort_by_device(ev, tgt_events);
    std::map<int, std::vector<AllocPair>> device_allocs_events;
    for (const AllocPair& p : alloc_events) device_allocs_events[ev[(size_t)p.alloc].dst_dev].push_back(p);

    int num_devices = 0;
    for (auto& kv : device_tgt_events) num_devices = std::max(num_devices, kv.first + 1);
    for (auto& kv : device_allocs_events) num_devices = std::max(num_devices, kv.first + 1);

    for (int dev_idx = 0; dev_idx < num_devices; ++dev_idx) {
        const std::vector<u64>& tgt = device_tgt_events[dev_idx];
        const std::vector<AllocPair>& allocs = device_allocs_events[dev_idx];
        size_t tgt_idx = 0;
        for (const AllocPair& p : allocs) {
            const Event& alloc_event = ev[(size_t)p.alloc];
            u64 delete_end = p.del == NONE ? trace_end : ev[(size_t)p.del].t_end_ns;
            while (tgt_idx < tgt.size() && ev[(size_t)tgt[tgt_idx]].t_end_ns < alloc_event.t_start_ns) {
                tgt_idx++;
            }
            if (tgt_idx == tgt.size() || ev[(size_t)tgt[tgt_idx]].t_start_ns > delete_end) {
                u64 ns = duration(alloc_event) + (p.del == NONE ? 0 : duration(ev[(size_t)p.del]));
                out.findings.push_back(make_finding(ev, F_UA, p.alloc, p.del, alloc_event.bytes, ns));
            }
        }
    }
}

// Algorithm 5, FindUnusedTransfers, over to-device transfers.  Per device a
// monotone kernel pointer; passing a kernel clears the candidate map; a
// transfer after the last kernel is unused; a transfer that starts before
// the current kernel overwrites (and flags) the previous candidate from the
// same host address; a transfer overlapping a kernel clears the candidates.
void find_unused_transfers(const std::vector<Event>& ev, const std::vector<u64>& tgt_events,
                           const std::vector<u64>& to_dev_events, Out& out) {
    std::map<int, std::vector<u64>> device_tgt_events = sort_by_device(ev, tgt_events);
    std::map<int, std::vector<u64>> device_tx_events = sort_by_device(ev, to_dev_events);
    int num_devices = 0;
    for (auto& kv : device_tgt_events) num_devices = std::max(num_devices, kv.first + 1);
    for (auto& kv : device_tx_events) num_devices = std::max(num_devices, kv.first + 1);

    for (int dev_idx = 0; dev_idx < num_devices; ++dev_idx) {
        const std::vector<u64>& tgt = device_tgt_events[dev_idx];
        const std::vector<u64>& txs = device_tx_events[dev_idx];
        size_t tgt_idx = 0;
        std::map<u64, u64> candidates;
        for (u64 txi : txs) {
            const Event& tx = ev[(size_t)txi];
            while (tgt_idx < tgt.size() && ev[(size_t)tgt[tgt_idx]].t_end_ns < tx.t_start_ns) {
                tgt_idx++;
                candidates.clear();
            }
            if (tgt_idx == tgt.size()) {
                // transfer occurs after the last active kernel
                out.findings.push_back(make_finding(ev, F_UT, txi, NONE, tx.bytes, duration(tx)));
            } else if (ev[(size_t)tgt[tgt_idx]].t_start_ns > tx.t_start_ns) {
                // transfer does not overlap an active kernel
                auto it = candidates.find(tx.host_addr);
                if (it != candidates.end()) {
                    const Event& cand = ev[(size_t)it->second];
                    out.findings.push_back(
                        make_finding(ev, F_UT, it->second, txi, cand.bytes, duration(cand)));
                }
                candidates[tx.host_addr] = txi;
            } else {
                candidates.clear();
            }
        }
    }
}

int analyze(const std::vector<Event>& ev, const std::vector<Content>& content, Out& out,
            Summary& sum) {
    std::memset(&sum, 0, sizeof sum);
    sum.n_events = ev.size();

    // Validation: the lowest offending index decides; a malformed record
    // wins over an out-of-order start time at the same index.
    for (u64 i = 0; i < ev.size(); ++i) {
        if (!record_ok(ev[(size_t)i])) return S_ERR_MALFORMED;
        if (i > 0 && ev[(size_t)i].t_start_ns < ev[(size_t)i - 1].t_start_ns) return S_ERR_UNSORTED;
    }

    std::vector<u64> data_op_events, to_dev_events, tgt_events;
    u64 begin = NONE, end = 0;
    for (u64 i = 0; i < ev.size(); ++i) {
        const Event& e = ev[(size_t)i];
        if (is_transfer(e)) data_op_events.push_back(i);
        if (e.kind == K_TO_DEV) to_dev_events.push_back(i);
        if (e.kind == K_KERNEL) tgt_events.push_back(i);
        if (e.kind == K_ALLOC) sum.n_allocs++;
        if (e.kind == K_DELETE) sum.n_deletes++;
        begin = std::min(begin, e.t_start_ns);
        end = std::max(end, e.t_end_ns);
    }
    if (ev.empty()) begin = 0;
    sum.n_transfers = data_op_events.size();
    sum.n_kernels = tgt_events.size();
    sum.trace_begin_ns = begin;
    sum.trace_end_ns = end;
    sum.trace_span_ns = end - begin;

    std::vector<AllocPair> pairs;
    std::vector<u64> unpaired;
    get_alloc_delete_pairs(ev, pairs, unpaired, sum.n_unmatched_deletes);
    sum.n_pairs = pairs.size();
    sum.n_unpaired_allocs = unpaired.size();

    find_duplicate_transfers(ev, content, data_op_events, out);
    find_round_trips(ev, content, data_op_events, out);
    find_repeated_allocs(ev, pairs, out);
    find_unused_allocs(ev, tgt_events, pairs, unpaired, end, out);
    find_unused_transfers(ev, tgt_events, to_dev_events, out);

    // Deliver findings ordered by (kind, event index).
    std::sort(out.findings.begin(), out.findings.end(), [](const Finding& l, const Finding& r) {
        if (l.kind != r.kind) return l.kind < r.kind;
        return l.event < r.event;
    });

    // Totals per kind and the union of wasted events (Sec. 7.6 estimate).
    std::vector<char> wasted(ev.size(), 0);
    std::map<u64, u64> delete_of_alloc;
    for (const AllocPair& p : pairs) delete_of_alloc[p.alloc] = p.del;
    for (const Finding& f : out.findings) {
        sum.count[f.kind]++;
        sum.wasted_bytes[f.kind] += f.wasted_bytes;
        sum.wasted_ns[f.kind] += f.wasted_ns;
        switch (f.kind) {
            case F_DD:
            case F_UT:
                wasted[(size_t)f.event] = 1;
                break;
            case F_RT:
                wasted[(size_t)f.partner] = 1;
                break;
            case F_RA:
                wasted[(size_t)f.event] = 1;
                wasted[(size_t)delete_of_alloc[f.event]] = 1;
                break;
            case F_UA:
                wasted[(size_t)f.event] = 1;
                if (f.partner != NONE) wasted[(size_t)f.partner] = 1;
                break;
        }
    }
    for (u64 i = 0; i < ev.size(); ++i)
        if (wasted[(size_t)i]) sum.saved_ns += duration(ev[(size_t)i]);
    sum.speedup_num = sum.trace_span_ns;
    sum.speedup_den = sum.trace_span_ns > sum.saved_ns ? sum.trace_span_ns - sum.saved_ns : 0;
    return S_OK;
}

void site_table(const std::vector<Finding>& findings, std::vector<SiteRow>& rows) {
    std::map<std::pair<int, u32>, SiteRow> agg;
    for (const Finding& f : findings) {
        std::pair<int, u32> key(f.kind, f.site);
        SiteRow& r = agg[key];
        r.site = f.site;
        r.kind = f.kind;
        r.count++;
        r.wasted_bytes += f.wasted_bytes;
        r.wasted_ns += f.wasted_ns;
    }
    for (auto& kv : agg) rows.push_back(kv.second);  // ordered by (kind, site)
}

int run(const Event* events, u64 n, const std::vector<Content>* override_content, Finding* items,
        u64 capacity, u64* count, Summary* summary, SiteRow* sites, u64 site_capacity,
        u64* n_sites) {
    std::vector<Event> ev(events, events + n);
    std::vector<Content> content(ev.size());
    for (u64 i = 0; i < n; ++i) {
        if (override_content) {
            content[(size_t)i] = (*override_content)[(size_t)i];
        } else {
            content[(size_t)i].a = ev[(size_t)i].fp_lo;
            content[(size_t)i].b = ev[(size_t)i].fp_hi;
        }
    }
    Out out;
    Summary sum;
    int status = analyze(ev, content, out, sum);
    if (status != S_OK) {
        std::memset(summary, 0, sizeof(Summary));
        *count = 0;
        *n_sites = 0;
        return status;
    }
    *summary = sum;
    *count = out.findings.size();
    for (u64 i = 0; i < out.findings.size() && i < capacity; ++i) items[i] = out.findings[(size_t)i];
    std::vector<SiteRow> rows;
    site_table(out.findings, rows);
    *n_sites = rows.size();
    for (u64 i = 0; i < rows.size() && i < site_capacity; ++i) sites[i] = rows[(size_t)i];
    if (out.findings.size() > capacity || rows.size() > site_capacity) return S_WARN_TRUNCATED;
    return S_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C interface (loaded with ctypes by the tests and the benchmark baseline)
// ---------------------------------------------------------------------------

extern "C" {

// FP128 v1 of `len` bytes at `data`; out[0] = low half, out[1] = high half.
void orc_fp128(const uint8_t* data, uint64_t len, uint64_t* out) {
    U128 h = fp128(data, len);
    out[0] = h.x;
    out[1] = h.y;
}

// FP128 of n buffers laid out back to back in `arena` (buffer i starts at
// offsets[i] and has sizes[i] bytes).
void orc_fp128_many(const uint8_t* arena, const uint64_t* offsets, const uint64_t* sizes,
                    uint64_t n, uint64_t* out) {
    for (uint64_t i = 0; i < n; ++i) {
        U128 h = fp128(arena + offsets[i], sizes[i]);
        out[2 * i] = h.x;
        out[2 * i + 1] = h.y;
    }
}

// Exposed pieces of the hash, for the invariant tests.
void orc_constant(int i, uint64_t* out) { *out = K().c[i]; }
void orc_splitmix64(uint64_t seed, uint64_t i, uint64_t* out) { *out = splitmix64_output(seed, i); }
void orc_chunk_leaf(const uint8_t* p, uint64_t r, uint64_t* out) {
    U128 h = chunk_leaf(p, r);
    out[0] = h.x;
    out[1] = h.y;
}
// State of lane l after its Feistel finish, for the chunk at p with r valid
// bytes (1..4096); out[0] = a chain, out[1] = b chain.
void orc_lane_state(const uint8_t* p, uint64_t r, int l, uint64_t* out) {
    uint8_t padded[CHUNK];
    pad_chunk(p, r, padded);
    U128 s = lane_state(padded, l);
    out[0] = s.x;
    out[1] = s.y;
}
void orc_tree_node(const uint64_t* left, const uint64_t* right, uint64_t count, uint64_t* out) {
    U128 l = {left[0], left[1]}, r = {right[0], right[1]};
    U128 h = tree_node(l, r, count);
    out[0] = h.x;
    out[1] = h.y;
}
void orc_mix128(int which, const uint64_t* in, uint64_t* out) {
    U128 s = {in[0], in[1]};
    U128 h = which == 0 ? mix_Q(s) : which == 1 ? mix_P(s) : mix_Z(s);
    out[0] = h.x;
    out[1] = h.y;
}
void orc_chain_step(int which, uint64_t v, uint64_t* out) {
    *out = which == 0 ? chain_step(v, K().odd(0), K().odd(1)) : chain_step(v, K().odd(2), K().odd(3));
}

// Algorithms 1-5 over an event log; fingerprints are taken from the records.
int orc_analyze(const void* events, uint64_t n, void* items, uint64_t capacity, uint64_t* count,
                void* summary, void* sites, uint64_t site_capacity, uint64_t* n_sites) {
    if (n > 0 && !events) return S_ERR_INVALID_ARG;
    return run((const Event*)events, n, nullptr, (Finding*)items, capacity, count,
               (Summary*)summary, (SiteRow*)sites, site_capacity, n_sites);
}

// Collision-check ("brute force") mode: content equality is decided by
// comparing the transferred bytes (and their lengths), not the fingerprint.
// payloads[i] points at event i's bytes (ignored for non-transfers).
int orc_analyze_bruteforce(const void* events, uint64_t n, const uint8_t* const* payloads,
                           void* items, uint64_t capacity, uint64_t* count, void* summary,
                           void* sites, uint64_t site_capacity, uint64_t* n_sites) {
    const Event* ev = (const Event*)events;
    std::vector<Content> content((size_t)n);
    std::vector<u64> reps;  // representative event of each distinct payload
    for (u64 i = 0; i < n; ++i) {
        content[(size_t)i].a = NONE;
        content[(size_t)i].b = i;
        if (!is_transfer(ev[i])) continue;
        bool found = false;
        for (u64 r : reps) {
            if (ev[r].bytes == ev[i].bytes &&
                std::memcmp(payloads[r], payloads[i], (size_t)ev[i].bytes) == 0) {
                content[(size_t)i] = content[(size_t)r];
                found = true;
                break;
            }
        }
        if (!found) {
            content[(size_t)i].a = 0;
            content[(size_t)i].b = reps.size();
            reps.push_back(i);
        }
    }
    return run(ev, n, &content, (Finding*)items, capacity, count, (Summary*)summary,
               (SiteRow*)sites, site_capacity, n_sites);
}

}  // extern "C"
