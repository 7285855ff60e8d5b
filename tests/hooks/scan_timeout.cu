// scan_timeout.cu -- test hook: runs the library's single-pass scan with its
// tile counter advanced past tile 0, so the block holding tile 1 waits for a
// status word that no block writes.  The wait is bounded: the kernel must
// end, set the fault word, and leave the context usable for a normal scan.
#include <cuda_runtime.h>

#include <vector>

#include "prims.cuh"

extern "C" int scan_timeout_case(uint32_t* fault_out, uint32_t* correct_after) {
    using namespace odp::prim;
    const uint32_t n = 2 * SCAN_TILE;  // tiles 0 and 1
    const size_t words = scan_tmp_words(n) + 16;
    uint32_t *in = nullptr, *out = nullptr, *tmp = nullptr, *fault = nullptr;
    if (cudaMalloc(&in, 4ull * n) != cudaSuccess || cudaMalloc(&out, 4ull * n) != cudaSuccess ||
        cudaMalloc(&tmp, 4 * words) != cudaSuccess || cudaMalloc(&fault, 4) != cudaSuccess)
        return 1;
    std::vector<uint32_t> h(n, 1u);
    cudaMemcpy(in, h.data(), 4ull * n, cudaMemcpyHostToDevice);
    cudaMemset(tmp, 0, 4 * words);
    cudaMemset(fault, 0, 4);
    const uint32_t one = 1;
    cudaMemcpy(tmp, &one, 4, cudaMemcpyHostToDevice);  // tile counter: tile 0 is never taken
    scan_chained<<<2, SCAN_THREADS>>>(in, out, nullptr, n, nullptr, tmp, fault);
    if (cudaDeviceSynchronize() != cudaSuccess) return 2;
    cudaMemcpy(fault_out, fault, 4, cudaMemcpyDeviceToHost);
    // the same scan from a clean scratch gives 0, 1, 2, ...
    cudaMemset(tmp, 0, 4 * words);
    cudaMemset(fault, 0, 4);
    scan_chained<<<2, SCAN_THREADS>>>(in, out, nullptr, n, nullptr, tmp, fault);
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;
    cudaMemcpy(h.data(), out, 4ull * n, cudaMemcpyDeviceToHost);
    uint32_t f = 0;
    cudaMemcpy(&f, fault, 4, cudaMemcpyDeviceToHost);
    bool ok = f == 0;
    for (uint32_t i = 0; i < n; ++i) ok &= h[i] == i;
    *correct_after = ok ? 1u : 0u;
    cudaFree(in);
    cudaFree(out);
    cudaFree(tmp);
    cudaFree(fault);
    return 0;
}
