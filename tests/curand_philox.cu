// Test helper: evaluates cuRAND's Philox4x32-10 (curand_Philox4x32_10) on the
// (counter, key) pairs of an input file, to pin the oracle's generator against
// an independent library implementation. Usage: curand_philox IN OUT N
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <curand_kernel.h>

__global__ void k_philox(const uint4* c, const uint2* k, uint4* o, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = curand_Philox4x32_10(c[i], k[i]);
}

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    const int n = atoi(argv[3]);
    std::vector<unsigned> in(6 * (size_t)n), out(4 * (size_t)n);
    FILE* f = fopen(argv[1], "rb");
    if (!f || fread(in.data(), 4, in.size(), f) != in.size()) return 3;
    fclose(f);
    uint4 *dc, *dout;
    uint2* dk;
    if (cudaMalloc(&dc, 16 * (size_t)n) || cudaMalloc(&dk, 8 * (size_t)n) || cudaMalloc(&dout, 16 * (size_t)n))
        return 4;
    cudaMemcpy(dc, in.data(), 16 * (size_t)n, cudaMemcpyHostToDevice);
    cudaMemcpy(dk, in.data() + 4 * (size_t)n, 8 * (size_t)n, cudaMemcpyHostToDevice);
    k_philox<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
    if (cudaMemcpy(out.data(), dout, 16 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess) return 5;
    f = fopen(argv[2], "wb");
    fwrite(out.data(), 4, out.size(), f);
    fclose(f);
    return 0;
}
