// Layout conversions on the device between the caller's row-major L x L
// bytes and the two colour planes (Sec. 3.3: white and black sites packed
// into separate arrays), plus the range check of uploaded spins.  They run
// on a device copy of the caller's buffer, so a state moves between host and
// device as one contiguous copy and is never touched byte by byte on the
// host.
//
// Row i of the row-major lattice holds, at column j = 2x + p, the site that
// sits at byte x of row i of the plane of colour (i + p) % 2: even rows
// interleave (white, black), odd rows (black, white).  A thread converts 32
// row-major bytes, i.e. 16 sites of each plane.  The conversions work on a
// block of nrows rows that starts at an even lattice row (the whole lattice,
// or the rows a row strip owns).
#include <algorithm>

#include "internal.cuh"

namespace potts {

namespace {

constexpr int kLayoutThreads = 256;

// Smallest index of a byte >= q in in[0, n) (n a multiple of 16), into *bad
// (which starts at ~0).
__global__ void check_spins_kernel(const uint8_t *in, int64_t n, uint32_t q,
                                   unsigned long long *bad) {
  const int64_t nv = n / 16;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(in) + v);
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (((words[k] >> (8 * b)) & 0xFFu) >= q) {
          atomicMin(bad, (unsigned long long)(v * 16 + 4 * k + b));
        }
      }
    }
  }
}

template <int LAY>
__global__ void rowmajor_to_planes_kernel(const uint8_t *in, int32_t L,
                                          int32_t nrows, uint8_t *white,
                                          uint8_t *black) {
  const int32_t H = L / 2, nch = H / 16;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nrows * nch) return;
  const int32_t i = (int32_t)(t / nch), c = (int32_t)(t - (int64_t)i * nch);
  const uint4 *src = reinterpret_cast<const uint4 *>(in + (int64_t)i * L) +
                     2 * c;
  const uint4 a = __ldcs(src), b = __ldcs(src + 1);
  const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint32_t ev[4], od[4];  // sites at even / odd columns
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ev[k] = __byte_perm(w[2 * k], w[2 * k + 1], 0x6420u);
    od[k] = __byte_perm(w[2 * k], w[2 * k + 1], 0x7531u);
  }
  const bool even_row = (i & 1) == 0;
  uint32_t *W = even_row ? ev : od, *B = even_row ? od : ev;
  if constexpr (LAY == kLayoutU4) {
    const int64_t o = (int64_t)i * (H / 2) + 8 * c;
    __stcs(reinterpret_cast<uint2 *>(white + o),
           make_uint2(pack8(W[0], W[1]), pack8(W[2], W[3])));
    __stcs(reinterpret_cast<uint2 *>(black + o),
           make_uint2(pack8(B[0], B[1]), pack8(B[2], B[3])));
  } else {
    const int64_t o = (int64_t)i * H + 16 * c;
    __stcs(reinterpret_cast<uint4 *>(white + o),
           make_uint4(W[0], W[1], W[2], W[3]));
    __stcs(reinterpret_cast<uint4 *>(black + o),
           make_uint4(B[0], B[1], B[2], B[3]));
  }
}

template <int LAY>
__global__ void planes_to_rowmajor_kernel(const uint8_t *white,
                                          const uint8_t *black, int32_t L,
                                          int32_t nrows, uint8_t *out) {
  const int32_t H = L / 2, nch = H / 16;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nrows * nch) return;
  const int32_t i = (int32_t)(t / nch), c = (int32_t)(t - (int64_t)i * nch);
  uint32_t W[4], B[4];
  if constexpr (LAY == kLayoutU4) {
    const int64_t o = (int64_t)i * (H / 2) + 8 * c;
    const uint2 pw = __ldcs(reinterpret_cast<const uint2 *>(white + o));
    const uint2 pb = __ldcs(reinterpret_cast<const uint2 *>(black + o));
    unpack8(pw.x, W[0], W[1]);
    unpack8(pw.y, W[2], W[3]);
    unpack8(pb.x, B[0], B[1]);
    unpack8(pb.y, B[2], B[3]);
  } else {
    const int64_t o = (int64_t)i * H + 16 * c;
    const uint4 pw = __ldcs(reinterpret_cast<const uint4 *>(white + o));
    const uint4 pb = __ldcs(reinterpret_cast<const uint4 *>(black + o));
    W[0] = pw.x; W[1] = pw.y; W[2] = pw.z; W[3] = pw.w;
    B[0] = pb.x; B[1] = pb.y; B[2] = pb.z; B[3] = pb.w;
  }
  const bool even_row = (i & 1) == 0;
  const uint32_t *E = even_row ? W : B, *O = even_row ? B : W;
  uint32_t r[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    r[2 * k] = __byte_perm(E[k], O[k], 0x5140u);
    r[2 * k + 1] = __byte_perm(E[k], O[k], 0x7362u);
  }
  uint4 *dst = reinterpret_cast<uint4 *>(out + (int64_t)i * L) + 2 * c;
  __stcs(dst, make_uint4(r[0], r[1], r[2], r[3]));
  __stcs(dst + 1, make_uint4(r[4], r[5], r[6], r[7]));
}

unsigned grid_for(int64_t threads) {
  return (unsigned)((threads + kLayoutThreads - 1) / kLayoutThreads);
}

}  // namespace

cudaError_t launch_check_spins(const uint8_t *in, int64_t n, uint32_t q,
                               unsigned long long *bad, cudaStream_t st) {
  if (n % 16) return cudaErrorInvalidValue;
  const int64_t nv = n / 16;
  const unsigned grid =
      (unsigned)std::min<int64_t>(grid_for(nv), 152 * 16);
  check_spins_kernel<<<grid, kLayoutThreads, 0, st>>>(in, n, q, bad);
  return cudaGetLastError();
}

cudaError_t launch_rowmajor_to_planes(const uint8_t *in, int32_t L,
                                      int32_t nrows, uint32_t layout,
                                      uint8_t *white, uint8_t *black,
                                      cudaStream_t st) {
  if (L % 32) return cudaErrorInvalidValue;
  const unsigned grid = grid_for((int64_t)nrows * (L / 32));
  if (layout == kLayoutU4)
    rowmajor_to_planes_kernel<kLayoutU4>
        <<<grid, kLayoutThreads, 0, st>>>(in, L, nrows, white, black);
  else
    rowmajor_to_planes_kernel<kLayoutU8>
        <<<grid, kLayoutThreads, 0, st>>>(in, L, nrows, white, black);
  return cudaGetLastError();
}

cudaError_t launch_planes_to_rowmajor(const uint8_t *white,
                                      const uint8_t *black, int32_t L,
                                      int32_t nrows, uint32_t layout,
                                      uint8_t *out, cudaStream_t st) {
  if (L % 32) return cudaErrorInvalidValue;
  const unsigned grid = grid_for((int64_t)nrows * (L / 32));
  if (layout == kLayoutU4)
    planes_to_rowmajor_kernel<kLayoutU4>
        <<<grid, kLayoutThreads, 0, st>>>(white, black, L, nrows, out);
  else
    planes_to_rowmajor_kernel<kLayoutU8>
        <<<grid, kLayoutThreads, 0, st>>>(white, black, L, nrows, out);
  return cudaGetLastError();
}

// Device staging buffer of n bytes on the stream's memory pool, copy of the
// planes in row-major order, copy to the caller's host buffer.
int download_rowmajor(const uint8_t *white, const uint8_t *black, int32_t L,
                      int32_t nrows, uint32_t layout, uint8_t *out_LxL,
                      cudaStream_t st) {
  const size_t n = (size_t)nrows * (size_t)L;
  uint8_t *stage = nullptr;
  if (cudaMallocAsync(&stage, n, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(POTTS_ENOMEM, "device staging buffer of %zu bytes", n);
  }
  cudaError_t e =
      launch_planes_to_rowmajor(white, black, L, nrows, layout, stage, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_LxL, stage, n, cudaMemcpyDeviceToHost, st);
  const cudaError_t ef = cudaFreeAsync(stage, st);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return fail(POTTS_ECUDA, "spin download failed: %s", cudaGetErrorString(e));
  return POTTS_OK;
}

// Copy of the caller's row-major spins to a device staging buffer, range
// check (every spin < q), then the split into the planes.  The planes are
// written only when every spin is in range.
int upload_rowmajor(const uint8_t *in_LxL, int32_t L, int32_t nrows,
                    uint32_t q, uint32_t layout, uint8_t *white,
                    uint8_t *black, cudaStream_t st) {
  const size_t n = (size_t)nrows * (size_t)L;
  uint8_t *stage = nullptr;
  if (cudaMallocAsync(&stage, n + 256, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(POTTS_ENOMEM, "device staging buffer of %zu bytes", n);
  }
  unsigned long long *d_bad = reinterpret_cast<unsigned long long *>(stage + n);
  unsigned long long bad = ~0ull;
  cudaError_t e = cudaMemcpyAsync(stage, in_LxL, n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0xFF, sizeof(bad), st);
  if (e == cudaSuccess && q < 256)
    e = launch_check_spins(stage, (int64_t)n, q, d_bad, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && bad == ~0ull)
    e = launch_rowmajor_to_planes(stage, L, nrows, layout, white, black, st);
  const cudaError_t ef = cudaFreeAsync(stage, st);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return fail(POTTS_ECUDA, "spin upload failed: %s", cudaGetErrorString(e));
  if (bad != ~0ull)
    return fail(POTTS_EINVAL, "spin %d at %llu is >= q = %u", in_LxL[bad],
                bad, q);
  return POTTS_OK;
}

}  // namespace potts
