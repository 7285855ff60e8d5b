// verify.cu -- odp_verify_fingerprints: the collision check of the paper's
// App. B (keep the transferred data and compare it wherever two fingerprints
// are equal) on the GPU.  Every transfer is compared byte for byte with the
// first transfer of the log carrying the same fingerprint; a difference in
// length or in any byte is a collision, i.e. a duplicate or round trip that
// the fingerprint would report falsely.
#include <algorithm>

#include "common.cuh"
#include "prims.cuh"

namespace odp {
namespace {

using prim::Key128;
using prim::NONE32;
using prim::Table;

struct VArgs {
    const uint8_t* ev;          // 64-byte records
    const void* const* payloads;
    uint32_t n;
    uint32_t* slot;
    Table tab;
    unsigned long long* n_collisions;
    uint8_t* flags;             // per event, may be null
};

__device__ __forceinline__ bool is_xfer(uint32_t kind) {
    return kind == ODP_TO_DEV || kind == ODP_FROM_DEV || kind == ODP_DEV_TO_DEV;
}

__device__ __forceinline__ uint32_t kind_of(const uint8_t* ev, uint32_t i) {
    return ev[64ull * i + 60];
}

__global__ void v_insert(VArgs a) {
    const uint32_t cap = *a.tab.cap_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        uint32_t s = NONE32;
        if (is_xfer(kind_of(a.ev, i))) {
            const uint64_t* r = reinterpret_cast<const uint64_t*>(a.ev + 64ull * i);
            s = prim::table_insert_min(a.tab, cap, Key128{r[5], r[6]}, i);
        }
        a.slot[i] = s;
    }
}

// One warp per transfer: compare with the first transfer of its fingerprint.
__global__ void v_compare(VArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < a.n; i += nw) {
        const uint32_t s = a.slot[i];
        if (s == NONE32) continue;
        const uint32_t rep = a.tab.slots[s].v;
        if (rep == i) {
            if (a.flags && lane == 0) a.flags[i] = 0;
            continue;
        }
        const uint64_t nb_i = reinterpret_cast<const uint64_t*>(a.ev + 64ull * i)[4];
        const uint64_t nb_r = reinterpret_cast<const uint64_t*>(a.ev + 64ull * rep)[4];
        const uint8_t* p = (const uint8_t*)a.payloads[i];
        const uint8_t* q = (const uint8_t*)a.payloads[rep];
        bool differ = nb_i != nb_r || (nb_i > 0 && (p == nullptr || q == nullptr));
        if (!differ && p != q) {
            const bool aligned = (((uintptr_t)p | (uintptr_t)q) & 15) == 0;
            const uint64_t words = aligned ? nb_i / 16 : 0;
            for (uint64_t w0 = 0; w0 < words && !differ; w0 += 32 * 4) {
                bool d = false;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint64_t w = w0 + u * 32 + lane;
                    if (w < words) {
                        const uint4 x = __ldcs(reinterpret_cast<const uint4*>(p) + w);
                        const uint4 y = __ldcs(reinterpret_cast<const uint4*>(q) + w);
                        d |= (x.x != y.x) | (x.y != y.y) | (x.z != y.z) | (x.w != y.w);
                    }
                }
                differ = __any_sync(ODP_FULL_MASK, d);
            }
            for (uint64_t b = words * 16 + lane; b < nb_i && !differ; b += 32 * 64) {
                bool d = false;
                for (uint64_t k = b; k < nb_i && k < b + 32 * 64; k += 32) d |= p[k] != q[k];
                differ = __any_sync(ODP_FULL_MASK, d);
            }
        }
        if (lane == 0) {
            if (a.flags) a.flags[i] = differ ? 1 : 0;
            if (differ) atomicAdd(a.n_collisions, 1ull);
        }
    }
}

__global__ void v_zero(unsigned long long* p) { *p = 0; }

}  // namespace
}  // namespace odp

extern "C" int odp_verify_fingerprints(const odp_event* events, const void* const* payloads,
                                       uint64_t n, unsigned long long* n_collisions,
                                       uint8_t* flags, cudaStream_t stream) {
    using namespace odp;
    if (!n_collisions) return ODP_ERR_INVALID_ARG;
    if (n > 0 && (!events || !payloads)) return ODP_ERR_INVALID_ARG;
    if (((uintptr_t)events & 15) != 0) return ODP_ERR_INVALID_ARG;
    if (n >= 0xFFFFFFF0ull) return ODP_ERR_UNSUPPORTED;
    v_zero<<<1, 1, 0, stream>>>(n_collisions);
    if (n == 0) return cuda_status(cudaGetLastError());
    const uint32_t nn = (uint32_t)n;
    uint32_t cap = 1024;
    while (cap < 2ull * nn) cap <<= 1;
    size_t bytes = 0;
    auto carve = [&](size_t sz) {
        size_t o = bytes;
        bytes = align_up(bytes + sz, 256);
        return o;
    };
    const size_t o_slot = carve(4ull * nn), o_slots = carve(sizeof(prim::Slot) * ((size_t)cap + 1)),
                 o_cap = carve(16);
    int st = ODP_OK;
    uint8_t* s = (uint8_t*)scratch_get(SLOT_AN_TABLE, bytes, stream, &st);
    if (!s) return st;
    VArgs a;
    a.ev = (const uint8_t*)events;
    a.payloads = payloads;
    a.n = nn;
    a.slot = (uint32_t*)(s + o_slot);
    a.tab.slots = (prim::Slot*)(s + o_slots);
    a.tab.cap_max = cap;
    a.tab.cap_dev = (uint32_t*)(s + o_cap);
    a.n_collisions = n_collisions;
    a.flags = flags;
    const int sms = device_sm_count();
    prim::table_clear<<<sms * 8, 256, 0, stream>>>(a.tab, nullptr, nn);
    v_insert<<<sms * 8, 256, 0, stream>>>(a);
    v_compare<<<sms * 8, 256, 0, stream>>>(a);
    return cuda_status(cudaGetLastError());
}
