// Throughput ceiling of the sweep's random-number work on this GPU.
//
// Kernel "philox": one Philox4x32-10 call per 4 sites with the sweep's
// counter layout (the library's own device generator).  Kernel "proposal":
// the same plus the four 32x32->64 products u*q that give the proposals and
// acceptance variates, packed as the colour pass packs them.  Neither reads
// or writes the lattice, so their rates bound the colour pass from above.
// Prints one JSON line with sites per second for each.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "../csrc/philox.cuh"

using potts::PhiloxKey;

__global__ void philox_only(uint32_t *sink, uint32_t key0, uint32_t key1,
                            uint32_t t_lo, uint32_t colour, int calls) {
  const PhiloxKey ks = potts::philox_schedule(key0, key1);
  uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) * (uint32_t)calls;
  uint32_t acc = 0;
  for (int i = 0; i < calls; i += 4) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 u = potts::philox10(g + k, t_lo, colour, 0u, ks);
      acc ^= u.x ^ u.y ^ u.z ^ u.w;
    }
    g += 4;
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void philox_proposal(uint32_t *sink, uint32_t key0, uint32_t key1,
                                uint32_t t_lo, uint32_t colour, uint32_t q,
                                int calls) {
  const PhiloxKey ks = potts::philox_schedule(key0, key1);
  uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) * (uint32_t)calls;
  uint32_t acc = 0, acc2 = 0;
  for (int i = 0; i < calls; i += 4) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 u = potts::philox10(g + k, t_lo, colour, 0u, ks);
      const uint64_t r0 = (uint64_t)u.x * q, r1 = (uint64_t)u.y * q;
      const uint64_t r2 = (uint64_t)u.z * q, r3 = (uint64_t)u.w * q;
      const uint32_t lo = __byte_perm((uint32_t)(r0 >> 32), (uint32_t)(r1 >> 32), 0x0040u);
      const uint32_t hi = __byte_perm((uint32_t)(r2 >> 32), (uint32_t)(r3 >> 32), 0x0040u);
      acc ^= __byte_perm(lo, hi, 0x5410u);
      acc2 += (uint32_t)r0 ^ (uint32_t)r1 ^ (uint32_t)r2 ^ (uint32_t)r3;
    }
    g += 4;
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc ^ acc2;
}

int main() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 128, blocks = sms * 16, calls = 64;
  uint32_t *sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * threads * 4) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double sites = 4.0 * blocks * threads * calls;
  double rate[2] = {0, 0};
  for (int kind = 0; kind < 2; ++kind) {
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
      cudaEventRecord(e0);
      if (kind == 0)
        philox_only<<<blocks, threads>>>(sink, 11u, 0u, 5u, 0u, calls);
      else
        philox_proposal<<<blocks, threads>>>(sink, 11u, 0u, 5u, 0u, 9u, calls);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    rate[kind] = sites / (best * 1e-3);
  }
  const cudaError_t err = cudaDeviceSynchronize();
  printf("{\"philox_sites_per_s\": %.4e, \"philox_proposal_sites_per_s\": %.4e, "
         "\"sms\": %d, \"status\": \"%s\"}\n",
         rate[0], rate[1], sms, cudaGetErrorString(err));
  cudaFree(sink);
  return err != cudaSuccess;
}
