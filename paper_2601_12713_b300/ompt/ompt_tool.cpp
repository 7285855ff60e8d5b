// ompt_tool.cpp -- an OMPT tool (OpenMP 5.1 tools interface, Sec. 4 of the
// specification) that turns a program's target data operations and kernel
// launches into mapping events for the serving loop, as the paper's profiler
// does with the same callbacks (Sec. 5: the EMI variants of the target,
// target-data-op and target-submit callbacks).  Every transfer is
// fingerprinted on the GPU when its bytes are in device memory (at the end
// of a transfer to the device, at the end of a transfer from or between
// devices), synchronously, so later kernels cannot change them first; the
// event then goes to odp_server_submit with ODP_EVENT_FP_GIVEN.  Each event
// is opened with odp_server_begin at its begin callback (which stamps its
// start), so the server's merge waits only for threads inside an operation
// and passes idle ones at once; an event that is not logged after all is
// cancelled.  At the end
// of the program the tool flushes the server, runs odp_analyze over the
// resident log and prints the counts; with ODP_OMPT_OUT=<prefix> it also
// writes <prefix>.events (the merged 64-byte records) and <prefix>.sites (one
// line per site id: the code address it stands for).
//
// The OMPT types and constants below are declared from the specification's
// interface tables (names, values and signatures).  Readings: for a delete,
// the device address is the operation's source; the host is the runtime's
// initial device (any negative device number too), mapped to -1.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "odp_ompt.h"

extern "C" {

typedef union ompt_data_t {
    uint64_t value;
    void* ptr;
} ompt_data_t;
typedef uint64_t ompt_id_t;
typedef void (*ompt_interface_fn_t)(void);
typedef ompt_interface_fn_t (*ompt_function_lookup_t)(const char* interface_function_name);
typedef void (*ompt_callback_t)(void);
typedef int (*ompt_set_callback_t)(int event, ompt_callback_t callback);
typedef int (*ompt_initialize_t)(ompt_function_lookup_t lookup, int initial_device_num,
                                 ompt_data_t* tool_data);
typedef void (*ompt_finalize_t)(ompt_data_t* tool_data);
typedef struct ompt_start_tool_result_t {
    ompt_initialize_t initialize;
    ompt_finalize_t finalize;
    ompt_data_t tool_data;
} ompt_start_tool_result_t;

}  // extern "C"

namespace {

// ompt_callbacks_t values
constexpr int OMPT_CB_TARGET_EMI = 33;
constexpr int OMPT_CB_TARGET_DATA_OP_EMI = 34;
constexpr int OMPT_CB_TARGET_SUBMIT_EMI = 35;
// ompt_set_result_t: at least "sometimes" means the callback will be dispatched
constexpr int OMPT_SET_SOMETIMES = 3;
// ompt_scope_endpoint_t
constexpr int OMPT_SCOPE_BEGIN = 1, OMPT_SCOPE_END = 2, OMPT_SCOPE_BEGINEND = 3;
// ompt_target_data_op_t (synchronous and asynchronous forms)
constexpr int OP_ALLOC = 1, OP_TO_DEVICE = 2, OP_FROM_DEVICE = 3, OP_DELETE = 4;
constexpr int OP_ALLOC_ASYNC = 17, OP_TO_DEVICE_ASYNC = 18, OP_FROM_DEVICE_ASYNC = 19,
              OP_DELETE_ASYNC = 20;

struct Tool {
    odp_server* server = nullptr;
    int host_device = -1;  // the runtime's number for the host (initial device)
    std::mutex site_mu;
    std::unordered_map<const void*, uint32_t> site_of;
    std::vector<const void*> sites;
    std::atomic<uint64_t> next_op{1};
    std::atomic<uint64_t> dropped{0};
};
Tool g_tool;

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

uint32_t site_id(const void* codeptr) {
    std::lock_guard<std::mutex> lk(g_tool.site_mu);
    auto it = g_tool.site_of.find(codeptr);
    if (it != g_tool.site_of.end()) return it->second;
    const uint32_t id = (uint32_t)std::min<size_t>(g_tool.sites.size(), ODP_MAX_SITES - 1);
    if (g_tool.sites.size() < ODP_MAX_SITES - 1) g_tool.sites.push_back(codeptr);
    g_tool.site_of.emplace(codeptr, id);
    return id;
}

int8_t dev_num(int d) { return d == g_tool.host_device || d < 0 ? (int8_t)-1 : (int8_t)d; }

// Per host thread: the operations between their begin and end callbacks,
// and the buffers of the synchronous fingerprint call.
struct ThreadState {
    std::unordered_map<uint64_t, uint64_t> begin_ns;  // host_op_id -> start
    cudaStream_t stream = nullptr;
    uint64_t* h_out = nullptr;   // pinned: lo, hi
    uint64_t* d_out = nullptr;   // device: lo, hi
    bool ready = false;
    ~ThreadState() {
        if (stream) cudaStreamDestroy(stream);
        if (h_out) cudaFreeHost(h_out);
        if (d_out) cudaFree(d_out);
    }
};
thread_local ThreadState t_state;

// FP128 of `bytes` bytes at device address p (synchronous); false on failure.
bool fingerprint_device(const void* p, uint64_t bytes, uint64_t* lo, uint64_t* hi) {
    ThreadState& t = t_state;
    if (!t.ready) {
        if (cudaStreamCreateWithFlags(&t.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaHostAlloc((void**)&t.h_out, 16, 0) != cudaSuccess ||
            cudaMalloc((void**)&t.d_out, 16) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        t.ready = true;
    }
    if (odp_fingerprint_one(p, bytes, (odp_fp128*)t.d_out, t.stream) != ODP_OK) return false;
    if (cudaMemcpyAsync(t.h_out, t.d_out, 16, cudaMemcpyDeviceToHost, t.stream) != cudaSuccess ||
        cudaStreamSynchronize(t.stream) != cudaSuccess)
        return false;
    *lo = t.h_out[0];
    *hi = t.h_out[1];
    return true;
}

// Start time of a new event, opened on the server so that the merge waits
// for it; every opened event is later submitted or cancelled.
uint64_t open_event() {
    uint64_t t = 0;
    if (g_tool.server && odp_server_begin(g_tool.server, &t) == ODP_OK) return t;
    return now_ns();
}

void drop(const odp_event& e) {
    if (g_tool.server) odp_server_cancel(g_tool.server, e.t_start_ns);
    g_tool.dropped.fetch_add(1);
}

void submit(const odp_event& e) {
    const void* payload = nullptr;
    if (!g_tool.server || odp_server_submit(g_tool.server, &e, &payload, 1) != ODP_OK) drop(e);
}

uint64_t begin_of(ompt_id_t* host_op_id, int endpoint) {
    if (endpoint != OMPT_SCOPE_BEGINEND && host_op_id) {
        auto& m = t_state.begin_ns;
        auto it = m.find(*host_op_id);
        if (it != m.end()) {
            const uint64_t b = it->second;
            m.erase(it);
            return b;
        }
    }
    return open_event();
}

void on_begin(ompt_id_t* host_op_id) {
    if (!host_op_id) return;
    *host_op_id = g_tool.next_op.fetch_add(1);
    t_state.begin_ns[*host_op_id] = open_event();
}

// Data operations that become events: allocations, deletes and transfers of
// a non-empty range with a device on at least one side.
bool logged_op(int optype, int src_device_num, int dest_device_num, size_t bytes) {
    switch (optype) {
        case OP_ALLOC:
        case OP_ALLOC_ASYNC:
        case OP_DELETE:
        case OP_DELETE_ASYNC:
            return true;
        case OP_TO_DEVICE:
        case OP_TO_DEVICE_ASYNC:
        case OP_FROM_DEVICE:
        case OP_FROM_DEVICE_ASYNC:
            return bytes != 0 && (dev_num(src_device_num) >= 0 || dev_num(dest_device_num) >= 0);
        default:
            return false;  // associate / disassociate: no data moves
    }
}

// target region: the device number rides in target_data for its kernels
void cb_target_emi(int /*kind*/, int endpoint, int device_num, ompt_data_t* /*task_data*/,
                   ompt_data_t* /*target_task_data*/, ompt_data_t* target_data,
                   const void* /*codeptr_ra*/) {
    if (endpoint == OMPT_SCOPE_BEGIN && target_data) target_data->value = (uint64_t)(device_num + 1);
}

void cb_target_data_op_emi(int endpoint, ompt_data_t* /*target_task_data*/,
                           ompt_data_t* /*target_data*/, ompt_id_t* host_op_id, int optype,
                           void* src_address, int src_device_num, void* dest_address,
                           int dest_device_num, size_t bytes, const void* codeptr_ra) {
    if (!logged_op(optype, src_device_num, dest_device_num, bytes)) return;
    if (endpoint == OMPT_SCOPE_BEGIN) {
        on_begin(host_op_id);
        return;
    }
    odp_event e{};
    e.t_start_ns = begin_of(host_op_id, endpoint);
    e.t_end_ns = std::max(now_ns(), e.t_start_ns);
    e.bytes = bytes;
    e.site_id = site_id(codeptr_ra);
    switch (optype) {
        case OP_ALLOC:
        case OP_ALLOC_ASYNC:
            e.kind = ODP_ALLOC;
            e.host_addr = (uint64_t)(uintptr_t)src_address;
            e.dev_addr = (uint64_t)(uintptr_t)dest_address;
            e.src_dev = -1;
            e.dst_dev = dev_num(dest_device_num);
            break;
        case OP_DELETE:
        case OP_DELETE_ASYNC:
            e.kind = ODP_DELETE;
            e.host_addr = (uint64_t)(uintptr_t)dest_address;
            e.dev_addr = (uint64_t)(uintptr_t)src_address;
            e.src_dev = -1;
            e.dst_dev = dev_num(src_device_num);
            break;
        case OP_TO_DEVICE:
        case OP_TO_DEVICE_ASYNC:
        case OP_FROM_DEVICE:
        case OP_FROM_DEVICE_ASYNC: {
            const bool to_dev = optype == OP_TO_DEVICE || optype == OP_TO_DEVICE_ASYNC;
            e.src_dev = dev_num(src_device_num);
            e.dst_dev = dev_num(dest_device_num);
            // the bytes in device memory: the destination of a transfer to a
            // device, else the source
            const void* dev_bytes = to_dev || e.src_dev < 0 ? dest_address : src_address;
            e.kind = e.src_dev < 0 ? ODP_TO_DEV : e.dst_dev < 0 ? ODP_FROM_DEV : ODP_DEV_TO_DEV;
            e.host_addr = (uint64_t)(uintptr_t)(e.kind == ODP_TO_DEV ? src_address : dest_address);
            e.dev_addr = (uint64_t)(uintptr_t)(e.kind == ODP_FROM_DEV ? src_address : dest_address);
            if (!fingerprint_device(dev_bytes, bytes, &e.fp_lo, &e.fp_hi)) {
                drop(e);
                return;
            }
            e.flags = ODP_EVENT_FP_GIVEN;
            break;
        }
        default:
            return;  // not reached: logged_op filtered the other kinds
    }
    submit(e);
}

void cb_target_submit_emi(int endpoint, ompt_data_t* target_data, ompt_id_t* host_op_id,
                          unsigned int /*requested_num_teams*/) {
    if (endpoint == OMPT_SCOPE_BEGIN) {
        on_begin(host_op_id);
        return;
    }
    odp_event e{};
    e.t_start_ns = begin_of(host_op_id, endpoint);
    e.t_end_ns = std::max(now_ns(), e.t_start_ns);
    e.kind = ODP_KERNEL;
    e.site_id = site_id(nullptr);  // the submit callback carries no code address
    e.src_dev = -1;
    e.dst_dev = target_data && target_data->value ? (int8_t)(target_data->value - 1) : 0;
    submit(e);
}

int tool_initialize(ompt_function_lookup_t lookup, int initial_device_num, ompt_data_t*) {
    g_tool.host_device = initial_device_num;
    auto set_cb = (ompt_set_callback_t)lookup("ompt_set_callback");
    if (!set_cb) return 0;
    odp_server_cfg cfg{};
    cfg.device = 0;
    cfg.n_slots = 2;
    cfg.max_events = 1u << 22;
    cfg.max_batch_events = 4096;
    cfg.max_producers = 256;
    cfg.watermark_timeout_us = 20000;
    cfg.batch_interval_us = 100;
    if (const char* s = std::getenv("ODP_OMPT_MAX_EVENTS")) cfg.max_events = std::strtoull(s, 0, 10);
    // the log capacity decides the device reservation; the budget is exactly it
    uint64_t need = 0;
    int rc = odp_server_bytes(&cfg, &need);
    if (rc == ODP_OK) {
        cfg.device_budget_bytes = need;
        rc = odp_server_create(&cfg, &g_tool.server);
    }
    if (rc != ODP_OK) {
        std::fprintf(stderr, "[odp] tool inactive: no server for a log of %llu events (%s)\n",
                     (unsigned long long)cfg.max_events, odp_status_string(rc));
        g_tool.server = nullptr;
        return 0;
    }
    const bool ok = set_cb(OMPT_CB_TARGET_EMI, (ompt_callback_t)cb_target_emi) >= OMPT_SET_SOMETIMES &&
                    set_cb(OMPT_CB_TARGET_DATA_OP_EMI, (ompt_callback_t)cb_target_data_op_emi) >=
                        OMPT_SET_SOMETIMES &&
                    set_cb(OMPT_CB_TARGET_SUBMIT_EMI, (ompt_callback_t)cb_target_submit_emi) >=
                        OMPT_SET_SOMETIMES;
    if (!ok) {
        odp_server_destroy(g_tool.server);
        g_tool.server = nullptr;
        return 0;
    }
    return 1;  // keep the tool active
}

void tool_finalize(ompt_data_t*) {
    if (!g_tool.server) return;
    odp_server_flush(g_tool.server);
    const odp_event* log = nullptr;
    uint64_t n = 0;
    odp_server_log(g_tool.server, &log, &n);
    const char* prefix = std::getenv("ODP_OMPT_OUT");
    if (n > 0) {
        const uint64_t cap = 6 * n + 64;
        odp_finding* items = nullptr;
        odp_site_row* rows = nullptr;
        uint64_t* small = nullptr;  // count, sites_count, status, summary
        const size_t small_bytes = 64 + sizeof(odp_summary);
        if (cudaMalloc(&items, sizeof(odp_finding) * cap) == cudaSuccess &&
            cudaMalloc(&rows, sizeof(odp_site_row) * 5 * ODP_MAX_SITES) == cudaSuccess &&
            cudaMalloc(&small, small_bytes) == cudaSuccess) {
            odp_findings out{};
            out.items = items;
            out.capacity = cap;
            out.count = small;
            out.sites = rows;
            out.sites_capacity = 5 * ODP_MAX_SITES;
            out.sites_count = small + 1;
            out.status = (int32_t*)(small + 2);
            out.summary = (odp_summary*)(small + 4);
            odp_summary sum{};
            int32_t status = 0;
            if (odp_analyze(log, n, &out, nullptr) == ODP_OK &&
                cudaMemcpy(&sum, out.summary, sizeof sum, cudaMemcpyDeviceToHost) == cudaSuccess &&
                cudaMemcpy(&status, out.status, 4, cudaMemcpyDeviceToHost) == cudaSuccess) {
                std::fprintf(stderr,
                             "[odp] %llu events: DD %llu RT %llu RA %llu UA %llu UT %llu "
                             "(status %d, %llu events dropped)\n",
                             (unsigned long long)n, (unsigned long long)sum.count[ODP_DD],
                             (unsigned long long)sum.count[ODP_RT],
                             (unsigned long long)sum.count[ODP_RA],
                             (unsigned long long)sum.count[ODP_UA],
                             (unsigned long long)sum.count[ODP_UT], status,
                             (unsigned long long)g_tool.dropped.load());
            }
        }
        cudaFree(items);
        cudaFree(rows);
        cudaFree(small);
        if (prefix) {
            std::vector<odp_event> host(n);
            std::string base(prefix);
            if (cudaMemcpy(host.data(), log, sizeof(odp_event) * n, cudaMemcpyDeviceToHost) ==
                cudaSuccess) {
                if (FILE* f = std::fopen((base + ".events").c_str(), "wb")) {
                    std::fwrite(host.data(), sizeof(odp_event), n, f);
                    std::fclose(f);
                }
            }
        }
    }
    if (prefix) {
        std::string base(prefix);
        if (FILE* f = std::fopen((base + ".sites").c_str(), "w")) {
            std::lock_guard<std::mutex> lk(g_tool.site_mu);
            for (size_t i = 0; i < g_tool.sites.size(); ++i)
                std::fprintf(f, "%zu %p\n", i, g_tool.sites[i]);
            std::fclose(f);
        }
    }
}

ompt_start_tool_result_t g_result = {tool_initialize, tool_finalize, {0}};

}  // namespace

extern "C" {

// Called by the OpenMP runtime at start-up (the tool is found through
// OMP_TOOL_LIBRARIES or by being linked into the program).
ompt_start_tool_result_t* ompt_start_tool(unsigned int /*omp_version*/,
                                          const char* /*runtime_version*/) {
    if (const char* s = std::getenv("ODP_OMPT_DISABLE"); s && *s && *s != '0') return nullptr;
    return &g_result;
}

// The tool's server (for a host program that wants the streamed findings).
odp_server* odp_ompt_server(void) { return g_tool.server; }

// Events the tool could not record (fingerprint or submit failures).
uint64_t odp_ompt_dropped(void) { return g_tool.dropped.load(); }

// Destroys the tool's server (after the runtime's finalize).
void odp_ompt_shutdown(void) {
    if (g_tool.server) odp_server_destroy(g_tool.server);
    g_tool.server = nullptr;
}

}  // extern "C"
