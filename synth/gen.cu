// gen.cu -- device-side fill of synthetic buffer contents (test and benchmark
// input only; no part of the analysed method).  Produces the same bytes as
// synth/content.py: word j of a "random" descriptor is SplitMix64 output
// (word_offset + j) of the stream seeded with `seed`; "page" tiles words
// 0..511; "zero" is all zero.  SplitMix64 follows its published definition
// (Steele, Lea, Flood, OOPSLA 2014).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ uint64_t sm64_out(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t word_of(int variant, uint64_t seed, uint64_t j) {
    if (variant == 1) return 0;
    if (variant == 2) return sm64_out(seed, j & 511);
    return sm64_out(seed, j);
}

// Fill `nbytes` bytes at dst (any alignment) with descriptor bytes starting
// at word `word_offset`.
__global__ void fill_kernel(uint8_t* dst, uint64_t nbytes, int variant, uint64_t seed,
                            uint64_t word_offset) {
    const uint64_t nwords = (nbytes + 7) / 8;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const bool aligned = ((uintptr_t)dst & 7) == 0;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nwords; j += stride) {
        uint64_t w = word_of(variant, seed, word_offset + j);
        if (aligned && 8 * j + 8 <= nbytes) {
            reinterpret_cast<uint64_t*>(dst)[j] = w;
        } else {
            for (int b = 0; b < 8 && 8 * j + b < nbytes; ++b) dst[8 * j + b] = (uint8_t)(w >> (8 * b));
        }
    }
}

// Batched fill: buffer i at base + offsets[i] with sizes[i] bytes and seed
// seeds[i] (random variant, word offset 0).  One block-stride loop per buffer
// chunk of 64 KiB.
__global__ void fill_many_kernel(uint8_t* base, const int64_t* offsets, const int64_t* sizes,
                                 const uint64_t* seeds, const int64_t* piece_buf,
                                 const int64_t* piece_first, int64_t n_pieces) {
    for (int64_t p = blockIdx.x; p < n_pieces; p += gridDim.x) {
        const int64_t i = piece_buf[p];
        const uint64_t w0 = (uint64_t)piece_first[p];  // first word of this piece
        const uint64_t nbytes = (uint64_t)sizes[i];
        const uint64_t nwords = (nbytes + 7) / 8;
        const uint64_t wend = w0 + 8192 < nwords ? w0 + 8192 : nwords;
        uint8_t* dst = base + offsets[i];
        const bool aligned = ((uintptr_t)dst & 7) == 0;
        for (uint64_t j = w0 + threadIdx.x; j < wend; j += blockDim.x) {
            uint64_t w = sm64_out(seeds[i], j);
            if (aligned && 8 * j + 8 <= nbytes) {
                reinterpret_cast<uint64_t*>(dst)[j] = w;
            } else {
                for (int b = 0; b < 8 && 8 * j + b < nbytes; ++b) dst[8 * j + b] = (uint8_t)(w >> (8 * b));
            }
        }
    }
}

}  // namespace

extern "C" {

int synth_fill(void* dst, uint64_t nbytes, int variant, uint64_t seed, uint64_t word_offset,
               cudaStream_t stream) {
    if (nbytes == 0) return 0;
    uint64_t nwords = (nbytes + 7) / 8;
    uint64_t blocks = (nwords + 255) / 256;
    if (blocks > 148 * 64) blocks = 148 * 64;
    fill_kernel<<<(unsigned)blocks, 256, 0, stream>>>((uint8_t*)dst, nbytes, variant, seed,
                                                       word_offset);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// pieces: (buffer index, first word) for every 64 KiB piece of every buffer
int synth_fill_many(void* base, const int64_t* offsets, const int64_t* sizes,
                    const uint64_t* seeds, const int64_t* piece_buf, const int64_t* piece_first,
                    int64_t n_pieces, cudaStream_t stream) {
    if (n_pieces == 0) return 0;
    int64_t blocks = n_pieces < 148 * 32 ? n_pieces : 148 * 32;
    fill_many_kernel<<<(unsigned)blocks, 256, 0, stream>>>((uint8_t*)base, offsets, sizes, seeds,
                                                           piece_buf, piece_first, n_pieces);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // extern "C"
