// Exhaustive check of the geometry update's division by w + 1 against the
// IEEE quotient: for every divisor b = 1..256 (w = 0..255), every significand
// of the numerator (2^23 values), both signs and exponents -40..8 (the range
// of fmaf(F, w, t) with |F|, |t| <= 1, w <= 255), div_by_weight(a, b, RN(1/b))
// must equal __fdiv_rn(a, b) bit for bit.  Prints the mismatch count and the
// first mismatch; exit status 0 when there is none.
#include <cstdio>
#include <cstdint>

#include "device_math.cuh"

__global__ void check(int e_lo, int e_hi, unsigned long long* bad, uint32_t* first) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;  // significand bits
    if (m >= (1u << 23)) return;
    unsigned long long nbad = 0;
    for (int w = 0; w < 256; ++w) {
        const float b = (float)(w + 1), y = __frcp_rn(b);
        for (int e = e_lo; e <= e_hi; ++e)
            for (int sgn = 0; sgn < 2; ++sgn) {
                const float a = __int_as_float((sgn << 31) | ((uint32_t)(e + 127) << 23) | m);
                const float q = tsdf::div_by_weight(a, b, y), r = __fdiv_rn(a, b);
                if (__float_as_uint(q) != __float_as_uint(r)) {
                    ++nbad;
                    if (atomicCAS(first, 0u, __float_as_uint(a)) == 0u) first[1] = (uint32_t)w;
                }
            }
    }
    if (nbad) atomicAdd(bad, nbad);
}

int main() {
    unsigned long long* bad;
    uint32_t* first;
    if (cudaMalloc(&bad, sizeof *bad) != cudaSuccess || cudaMalloc(&first, 2 * sizeof *first) != cudaSuccess) return 2;
    cudaMemset(bad, 0, sizeof *bad);
    cudaMemset(first, 0, 2 * sizeof *first);
    check<<<(1u << 23) / 256, 256>>>(-40, 8, bad, first);
    unsigned long long h = 0;
    uint32_t f[2] = {0, 0};
    if (cudaDeviceSynchronize() != cudaSuccess) return 2;
    cudaMemcpy(&h, bad, sizeof h, cudaMemcpyDeviceToHost);
    cudaMemcpy(f, first, sizeof f, cudaMemcpyDeviceToHost);
    std::printf("checked %llu quotients, %llu mismatches", 256ull * 49 * 2 * (1ull << 23), h);
    if (h) std::printf(" (first: a bits 0x%08x, w %u)", f[0], f[1]);
    std::printf("\n");
    return h ? 1 : 0;
}
