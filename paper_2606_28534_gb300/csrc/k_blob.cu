// k_blob.cu -- checks of a checkpoint blob on the device (paper Sec. 4.1: checkpoint/restart of
// the particle state), so that a restart from a large blob is bound by the host-to-device copy
// rather than by a host pass over the blob.
//
// k_blob_crc: the CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320, as zlib) register of every
// full 64 KB block of the blob, each from a zero register; the host joins them in order.  The CRC
// register update is linear over GF(2), so R(r, A || B) = Z^{|B|}(R(r, A)) xor R(0, B), with Z the
// update by one zero byte.  A warp takes a block: lane l the 2 KB piece l (slice-by-8 tables in
// shared memory, eight bytes per step), then the lanes' registers are joined in a tree of five
// levels with the operators Z^{2048 d}, d = 1, 2, 4, 8, 16 (32 x 32 matrices over GF(2), column i
// the image of bit i, made on the host).
//
// k_blob_ranges: every record's cell word and fraction (the snapshot's per-species arrays: u32
// cell words, then f64 fractions) in range: cell < N; the countdown pair 0 or, for a species with
// the null-collision countdown, 1 <= k <= 4095 with the candidate flag in bit 12; 0 <= f < 1.
#include "pic_internal.cuh"

namespace {

constexpr int CRC_BLOCK = 65536;        // bytes per warp
constexpr int CRC_PIECE = CRC_BLOCK / 32;  // bytes per lane
constexpr int CRC_TPB = 256;

__device__ __forceinline__ uint32_t gf2_apply_dev(const uint32_t* m, uint32_t v) {
  uint32_t r = 0u;
#pragma unroll 1
  for (int i = 0; v; ++i, v >>= 1)
    if (v & 1u) r ^= m[i];
  return r;
}

__global__ void __launch_bounds__(CRC_TPB) k_blob_crc(const unsigned char* __restrict__ p, unsigned long long nblocks,
                                                      const BlobCrcOps ops, uint32_t* __restrict__ out) {
  __shared__ uint32_t T[8][256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    uint32_t c = (uint32_t)i;
    for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : (c >> 1);
    T[0][i] = c;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    uint32_t c = T[0][i];
    for (int k = 1; k < 8; ++k) {
      c = T[0][c & 0xFFu] ^ (c >> 8);
      T[k][i] = c;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned long long warps = (unsigned long long)gridDim.x * (CRC_TPB / 32);
  for (unsigned long long b = (unsigned long long)blockIdx.x * (CRC_TPB / 32) + (threadIdx.x >> 5); b < nblocks;
       b += warps) {
    const uint4* q = reinterpret_cast<const uint4*>(p + b * CRC_BLOCK + (size_t)lane * CRC_PIECE);
    uint32_t c = 0u;
#pragma unroll 4
    for (int i = 0; i < CRC_PIECE / 16; ++i) {
      const uint4 v = q[i];
      uint32_t lo = v.x ^ c, hi = v.y;
      c = T[7][lo & 0xFFu] ^ T[6][(lo >> 8) & 0xFFu] ^ T[5][(lo >> 16) & 0xFFu] ^ T[4][lo >> 24] ^ T[3][hi & 0xFFu] ^
          T[2][(hi >> 8) & 0xFFu] ^ T[1][(hi >> 16) & 0xFFu] ^ T[0][hi >> 24];
      lo = v.z ^ c;
      hi = v.w;
      c = T[7][lo & 0xFFu] ^ T[6][(lo >> 8) & 0xFFu] ^ T[5][(lo >> 16) & 0xFFu] ^ T[4][lo >> 24] ^ T[3][hi & 0xFFu] ^
          T[2][(hi >> 8) & 0xFFu] ^ T[1][(hi >> 16) & 0xFFu] ^ T[0][hi >> 24];
    }
    // join: at level k, lane l (l % 2d == 0) takes its right neighbour's register l + d, whose
    // piece is 2048 d bytes long
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int d = 1 << k;
      const uint32_t r = __shfl_down_sync(0xFFFFFFFFu, c, d);
      if ((lane & (2 * d - 1)) == 0) c = gf2_apply_dev(ops.z[k], c) ^ r;
    }
    if (lane == 0) out[b] = c;
  }
}

__global__ void __launch_bounds__(256) k_blob_ranges(const unsigned char* __restrict__ cells,
                                                     const unsigned char* __restrict__ fracs, unsigned long long m, int N,
                                                     int mcc, unsigned int* __restrict__ bad) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  bool ok = true;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const uint32_t w = reinterpret_cast<const uint32_t*>(cells)[i];
    // the fractions follow 4 m bytes of cell words: 4-byte aligned only, so two 32-bit loads
    const uint32_t* fp = reinterpret_cast<const uint32_t*>(fracs + 8ull * i);
    const double f = __hiloint2double((int)fp[1], (int)fp[0]);
    const uint32_t pair = w >> PIC_CELL_BITS;
    const bool pair_ok =
        mcc ? (pair == 0u || (pair <= (PIC_NEXT_CAND | PIC_NEXT_KMAX) && (pair & PIC_NEXT_KMAX) != 0u)) : pair == 0u;
    if ((int)(w & PIC_CELL_MASK) >= N || !pair_ok || !(f >= 0.0 && f < 1.0)) ok = false;
  }
  if (__any_sync(0xFFFFFFFFu, !ok) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

}  // namespace

cudaError_t launch_blob_crc(const unsigned char* p, unsigned long long nblocks, const BlobCrcOps& ops, uint32_t* out,
                            cudaStream_t st) {
  if (nblocks == 0) return cudaSuccess;
  const unsigned long long ctas = (nblocks + CRC_TPB / 32 - 1) / (CRC_TPB / 32);
  k_blob_crc<<<(unsigned)(ctas < 4096ull ? ctas : 4096ull), CRC_TPB, 0, st>>>(p, nblocks, ops, out);
  return cudaGetLastError();
}

cudaError_t launch_blob_ranges(const unsigned char* cells, const unsigned char* fracs, unsigned long long m, int N,
                               int mcc, unsigned int* bad, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  const unsigned long long need = (m + 255) / 256;
  k_blob_ranges<<<(unsigned)(need < 4096ull ? need : 4096ull), 256, 0, st>>>(cells, fracs, m, N, mcc, bad);
  return cudaGetLastError();
}
