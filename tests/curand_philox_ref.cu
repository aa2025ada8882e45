// Test helper (built and run by tests/test_gpu_curand_pin.py): the site
// words of the Philox4x32-10 counter layout, computed on the GPU by
// cuRAND's device-side Philox4_32_10 generator, an implementation
// independent of the oracle's.
//
// cuRAND keys its generator with (seed mod 2^32, seed >> 32), puts the
// subsequence in counter words 2..3 and the offset / 4 in counter words
// 0..1; a state advanced by a multiple of 4 words returns the four words of
// Philox(counter, key) from curand4().  So the word of site k of colour
// (domain) c in sweep t is word k & 3 of curand4() after
// curand_init(seed, c | t_hi << 32, 0) and an advance of 4 (t_lo << 32 |
// k >> 2) words (taken in parts: skipahead counts words in 64 bits).
//
// Usage: curand_philox_ref <in.bin> <out.bin>; in: n records of four
// uint64 (seed, sweep, domain, k); out: n uint32 words.
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdint>
#include <cstdio>
#include <vector>

__global__ void site_words(const unsigned long long *in, uint32_t *out,
                           int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long seed = in[4 * i], sweep = in[4 * i + 1],
                           dom = in[4 * i + 2], k = in[4 * i + 3];
  const unsigned long long sub = dom | ((sweep >> 32) << 32);
  const unsigned long long blk = ((sweep & 0xFFFFFFFFull) << 32) | (k >> 2);
  curandStatePhilox4_32_10_t st;
  curand_init(seed, sub, 0ull, &st);
  // advance blk counter blocks: four times blk / 4, then blk % 4 (each
  // word count below 2^64)
  for (int j = 0; j < 4; ++j) skipahead(4ull * (blk >> 2), &st);
  skipahead(4ull * (blk & 3ull), &st);
  const uint4 r = curand4(&st);
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
  out[i] = w[k & 3];
}

int main(int argc, char **argv) {
  if (argc != 3) return 2;
  FILE *f = fopen(argv[1], "rb");
  if (!f) return 3;
  std::vector<unsigned long long> in;
  unsigned long long v[4];
  while (fread(v, sizeof(v), 1, f) == 1) in.insert(in.end(), v, v + 4);
  fclose(f);
  const int n = (int)(in.size() / 4);
  if (n == 0) return 4;
  unsigned long long *d_in = nullptr;
  uint32_t *d_out = nullptr;
  if (cudaMalloc(&d_in, in.size() * sizeof(in[0])) != cudaSuccess ||
      cudaMalloc(&d_out, (size_t)n * sizeof(uint32_t)) != cudaSuccess)
    return 5;
  cudaMemcpy(d_in, in.data(), in.size() * sizeof(in[0]),
             cudaMemcpyHostToDevice);
  site_words<<<(n + 255) / 256, 256>>>(d_in, d_out, n);
  std::vector<uint32_t> out((size_t)n);
  if (cudaMemcpy(out.data(), d_out, out.size() * sizeof(uint32_t),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return 6;
  cudaFree(d_in);
  cudaFree(d_out);
  FILE *g = fopen(argv[2], "wb");
  if (!g) return 7;
  fwrite(out.data(), sizeof(uint32_t), out.size(), g);
  fclose(g);
  return 0;
}
