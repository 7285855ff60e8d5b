// loadgen.cpp -- host threads that emit mapping events with Poisson arrivals
// (test and benchmark input for the serving loop; none of the analysed
// method's arithmetic).  Each thread runs map cycles (ALLOC, TO_DEV, KERNEL,
// FROM_DEV, DELETE) on its own host ranges; a transfer's payload is a view
// (offset, size) into a device-resident content pool, and resending a view
// resends unchanged content.  Random numbers: SplitMix64 (Steele, Lea,
// Flood 2014) as a counter-based generator, seeded per thread.
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

#pragma pack(push, 1)
struct Event {
    uint64_t t_start_ns, t_end_ns, host_addr, dev_addr, bytes, fp_lo, fp_hi;
    uint32_t site_id;
    uint8_t kind;
    int8_t src_dev, dst_dev;
    uint8_t flags;
};
#pragma pack(pop)
static_assert(sizeof(Event) == 64, "64-byte record");

enum { ALLOC = 1, TO_DEV = 2, FROM_DEV = 3, DELETE = 5, KERNEL = 6 };

typedef int (*submit_fn)(void* server, const void* events, const void* const* payloads, uint64_t n);
typedef int (*attach_fn)(void* server, uint64_t start_t_ns);
typedef int (*begin_fn)(void* server, uint64_t* t_start_ns);

struct Rng {
    uint64_t s, i = 0;
    explicit Rng(uint64_t seed) : s(seed) {}
    uint64_t next() {
        uint64_t z = s + (++i) * 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct View {
    uint64_t off, size;
};

struct Cfg {
    uint32_t n_threads;
    double events_per_s;
    double seconds;
    uint64_t seed;
    const uint8_t* pool;  // device address of the content pool
    uint64_t pool_bytes;
    uint64_t min_payload, max_payload;
};

struct Thread {
    std::vector<View> payload_of_seq;  // per submitted event (size 0: none)
    uint64_t submitted = 0;
    int rc = 0;
};

struct Gen {
    Cfg cfg;
    std::vector<Thread> th;
};

void producer(Gen* g, uint32_t k, void* server, submit_fn submit, attach_fn attach,
              begin_fn begin, std::atomic<bool>* go, std::atomic<uint32_t>* ready) {
    const Cfg& c = g->cfg;
    Thread& T = g->th[k];
    Rng r(c.seed ^ (0x5EED0000ull + k) * 0xD1342543DE82EF95ull);
    const double rate = c.events_per_s / c.n_threads;
    const uint64_t host_base = 0x7F00000000000000ull + ((uint64_t)k << 40);
    const uint64_t dev_base = 0x0000100000000000ull + ((uint64_t)k << 36);
    std::vector<View> sent;
    std::vector<std::pair<uint64_t, uint64_t>> freed;  // (host_addr, bytes)
    uint64_t dev_next = dev_base;
    const double lo = std::log((double)c.min_payload), hi = std::log((double)c.max_payload);
    auto rand_size = [&]() {
        return (uint64_t)std::exp(lo + r.uniform() * (hi - lo));
    };
    auto fresh_view = [&](uint64_t size) {
        uint64_t span = c.pool_bytes > size ? c.pool_bytes - size : 0;
        uint64_t off = (uint64_t)(r.uniform() * (double)span) & ~15ull;
        return View{off, size};
    };
    // register before the first event so the server's merge waits for us
    if (attach && attach(server, 0) < 0) T.rc = -1;
    ready->fetch_add(1);
    while (!go->load()) std::this_thread::yield();
    const uint64_t t_begin = now_ns();
    const uint64_t t_stop = t_begin + (uint64_t)(c.seconds * 1e9);
    double t_next = (double)t_begin;
    uint32_t site_enter = (uint32_t)(r.next() % 500), site_exit = (uint32_t)(r.next() % 500);
    auto emit = [&](Event e, const View* v) -> bool {
        t_next += -std::log(1.0 - r.uniform()) / rate * 1e9;  // exponential gap
        uint64_t now = now_ns();
        if ((double)now < t_next) {
            std::this_thread::sleep_for(std::chrono::nanoseconds((uint64_t)(t_next - (double)now)));
            now = now_ns();
        }
        if (now >= t_stop) return false;
        // with a begin call the server stamps the start (its clock is the
        // same steady clock)
        if (begin) {
            int rc = begin(server, &now);
            if (rc < 0) {
                T.rc = rc;
                return false;
            }
        }
        const uint64_t dur = e.t_end_ns;  // duration stashed by the caller
        e.t_start_ns = now;
        e.t_end_ns = now + dur;
        const void* payload = v ? (const void*)(c.pool + v->off) : nullptr;
        int rc = submit(server, &e, &payload, 1);
        if (rc < 0) {
            T.rc = rc;
            return false;
        }
        T.payload_of_seq.push_back(v ? *v : View{0, 0});
        ++T.submitted;
        return true;
    };
    auto xfer_ns = [](uint64_t bytes) { return 2000 + bytes * 1000 / 25000; };
    while (true) {
        Event e;
        std::memset(&e, 0, sizeof e);
        uint64_t host, bytes;
        const bool ra = !freed.empty() && r.uniform() < 0.05;
        if (ra) {
            auto f = freed[r.next() % freed.size()];
            host = f.first;
            bytes = f.second;
        } else {
            bytes = rand_size();
            host = host_base + ((r.next() % (1ull << 24)) << 12);
        }
        const uint64_t dev = dev_next;
        dev_next += (bytes + 4095) & ~4095ull;
        if (dev_next > dev_base + (1ull << 35)) dev_next = dev_base;
        // ALLOC
        e.kind = ALLOC; e.src_dev = -1; e.dst_dev = 0; e.host_addr = host; e.dev_addr = dev;
        e.bytes = bytes; e.site_id = site_enter; e.t_end_ns = 1000;
        if (!emit(e, nullptr)) break;
        // TO_DEV: 30 % resend an earlier view of the same size class
        View vin;
        bool dd = false;
        if (!sent.empty() && r.uniform() < 0.30) {
            vin = sent[r.next() % sent.size()];
            dd = true;
        } else {
            vin = fresh_view(bytes);
        }
        e.kind = TO_DEV; e.src_dev = -1; e.dst_dev = 0; e.bytes = vin.size;
        e.t_end_ns = xfer_ns(vin.size);
        if (!emit(e, &vin)) break;
        if (!dd) sent.push_back(vin);
        // KERNEL
        e.kind = KERNEL; e.src_dev = -1; e.dst_dev = 0; e.bytes = 0;
        e.t_end_ns = (uint64_t)(50000.0 * std::exp(r.uniform() * std::log(100.0)));
        if (!emit(e, nullptr)) break;
        // FROM_DEV: 10 % return the content unchanged (a round trip)
        View vout = r.uniform() < 0.10 ? vin : fresh_view(vin.size);
        e.kind = FROM_DEV; e.src_dev = 0; e.dst_dev = -1; e.bytes = vout.size;
        e.site_id = site_exit; e.t_end_ns = xfer_ns(vout.size);
        if (!emit(e, &vout)) break;
        // DELETE
        e.kind = DELETE; e.src_dev = -1; e.dst_dev = 0; e.bytes = bytes; e.t_end_ns = 1000;
        if (!emit(e, nullptr)) break;
        freed.emplace_back(host, bytes);
        if (freed.size() > 64) freed.erase(freed.begin());
        if (sent.size() > 256) sent.erase(sent.begin());
    }
}

}  // namespace

extern "C" {

void* synth_load_create(uint32_t n_threads, double events_per_s, double seconds, uint64_t seed,
                        const void* pool, uint64_t pool_bytes, uint64_t min_payload,
                        uint64_t max_payload) {
    Gen* g = new Gen();
    g->cfg = Cfg{n_threads, events_per_s, seconds, seed, (const uint8_t*)pool, pool_bytes,
                 min_payload, max_payload};
    g->th.resize(n_threads);
    return g;
}

// Runs all producer threads to completion; returns the number of events
// submitted, or a negative submit status.  `begin` may be null (events are
// then stamped with the thread's own clock at submit time).
int64_t synth_load_run(void* h, void* server, void* submit, void* attach, void* begin) {
    Gen* g = (Gen*)h;
    std::atomic<bool> go{false};
    std::atomic<uint32_t> ready{0};
    std::vector<std::thread> ts;
    for (uint32_t k = 0; k < g->cfg.n_threads; ++k)
        ts.emplace_back(producer, g, k, server, (submit_fn)submit, (attach_fn)attach,
                        (begin_fn)begin, &go, &ready);
    while (ready.load() < g->cfg.n_threads) std::this_thread::yield();
    go = true;
    for (auto& t : ts) t.join();
    int64_t total = 0;
    for (auto& T : g->th) {
        if (T.rc < 0) return T.rc;
        total += (int64_t)T.submitted;
    }
    return total;
}

// Payload view of event `seq` of producer thread `k` (size 0: no payload).
int synth_load_payload(void* h, uint32_t k, uint64_t seq, uint64_t* off, uint64_t* size) {
    Gen* g = (Gen*)h;
    if (k >= g->th.size() || seq >= g->th[k].payload_of_seq.size()) return -1;
    *off = g->th[k].payload_of_seq[seq].off;
    *size = g->th[k].payload_of_seq[seq].size;
    return 0;
}

uint32_t synth_load_thread_of(uint64_t host_addr) {
    return (uint32_t)((host_addr - 0x7F00000000000000ull) >> 40);
}

void synth_load_destroy(void* h) { delete (Gen*)h; }

}  // extern "C"
