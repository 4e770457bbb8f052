// k_sort.cu -- the arranger: per-cell counting sort with compaction (BIT1's "natural sorting",
// paper Sec. 2; the arrj/narrj arranger of Sec. 5.1).
//
// The per-cell particle counts come for free from the deposit of the step that precedes the
// sort (every live particle, births and source pairs included, was counted in its cell), so the
// sort is two launches:
//   k_sort_scan     one 8-CTA cluster per species: exclusive scan of the counts -> per-cell write
//                   cursors;
//                   records the old extent, sets the new one, pads the destination with DEAD
//                   cells and clears the counts;
//   k_sort_scatter  persistent tiles over the old arrays (both species): every live particle
//                   claims a slot in its cell with one warp-aggregated atomic per (warp, cell)
//                   group (__match_any_sync) and is copied to the other buffer.  Dead particles
//                   are dropped (compaction).
// The order inside a cell follows the atomic claims and is not reproducible; every per-particle
// result of the method depends only on the particle itself, the step and the field, so the state
// as a set of particles is reproducible, and snapshots are written in id order.
#include <cooperative_groups.h>

#include <cstring>

#include "pic_internal.cuh"

namespace cg = cooperative_groups;

namespace {

// One cluster of PIC_FIELD_CTAS CTAs per species: each CTA stages a contiguous segment of the
// counts in shared memory (coalesced), scans runs of consecutive cells per thread, and takes its
// offset from the CTA totals of the lower ranks through distributed shared memory.
// BATCH: clusters 2k and 2k + 1 scan species 0 and 1 of simulation k of an ensemble, with the
// parameters tab[k].
template <bool BATCH>
__global__ void __cluster_dims__(PIC_FIELD_CTAS, 1, 1) __launch_bounds__(1024, 1)
    k_sort_scan(const __grid_constant__ SortParams P0, const SortParams* __restrict__ tab) {
  extern __shared__ unsigned int cs[];
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long cta_tot;
  cg::cluster_group cluster = cg::this_cluster();
  const SortParams& P = BATCH ? tab[blockIdx.x / (2 * PIC_FIELD_CTAS)] : P0;
  const int s = BATCH ? (int)((blockIdx.x / PIC_FIELD_CTAS) & 1u) : (int)(blockIdx.x / PIC_FIELD_CTAS);
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int N = P.N;
  unsigned int* cnt = s ? P.cnt[1] : P.cnt[0];
  unsigned int* cur = s ? P.cursor[1] : P.cursor[0];
  const int seg = (N + PIC_FIELD_CTAS - 1) / PIC_FIELD_CTAS;
  const int a = rank * seg;
  const int len = max(0, min(seg, N - a));
  for (int i = tid; i < len; i += 1024) {
    cs[i] = cnt[a + i];
    cnt[a + i] = 0u;
  }
  __syncthreads();
  const int items = (len + 1023) / 1024;
  const int i0 = tid * items;
  unsigned long long own = 0ull;
  for (int k = 0; k < items; ++k) {
    const int i = i0 + k;
    if (i < len) own += cs[i];
  }
  unsigned long long incl = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (tid < 32) {
    unsigned long long v = warp_tot[tid];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += u;
    }
    warp_tot[tid] = v;
    if (tid == 31) cta_tot = v;
  }
  __syncthreads();
  cluster.sync();
  unsigned long long off = 0ull, total = 0ull;
#pragma unroll
  for (int r = 0; r < PIC_FIELD_CTAS; ++r) {
    const unsigned long long v = *cluster.map_shared_rank(&cta_tot, r);
    if (r < rank) off += v;
    total += v;
  }
  unsigned long long run = off + (w ? warp_tot[w - 1] : 0ull) + incl - own;
  for (int k = 0; k < items; ++k) {
    const int i = i0 + k;
    if (i < len) {
      const unsigned int c = cs[i];
      cs[i] = (unsigned int)run;
      run += c;
    }
  }
  __syncthreads();
  for (int i = tid; i < len; i += 1024) cur[a + i] = cs[i];
  if (rank == 0 && tid == 0) {
    Ctl* g = P.ctl;
    g->sort_total[s] = g->n_cur[s];  // old extent, read by the scatter
    if (total != g->n_live[s]) atomicOr(&g->error, ERR_DEVICE);
    const unsigned long long cap = s ? P.cap[1] : P.cap[0];
    unsigned long long pad = round_up4(total);
    if (pad > cap) {  // counts inconsistent with the capacity: flag, never write past the end
      atomicOr(&g->error, ERR_DEVICE);
      pad = cap;
    }
    int* dcell = s ? P.dst[1].cell : P.dst[0].cell;
    for (unsigned long long i = total; i < pad; ++i) dcell[i] = PIC_DEAD_CELL;
    if (P.defer)
      g->sort_new[s] = pad;
    else
      g->n_cur[s] = pad;
  }
  cluster.sync();  // keep the CTA totals alive until every rank has read them
}

template <int s>
__device__ __forceinline__ void scatter_tile(const SortParams& P, unsigned long long i0, bool have) {
  const Species32& A = P.src[s];
  const Species32& D = P.dst[s];
  unsigned int* cur = P.cursor[s];
  int c[PIC_PPT];
  float f[PIC_PPT], vx[PIC_PPT], vy[PIC_PPT], vz[PIC_PPT];
  unsigned long long id[PIC_PPT];
  if (have) {
    int4 c4 = *reinterpret_cast<const int4*>(A.cell + i0);
    float4 f4 = *reinterpret_cast<const float4*>(A.frac + i0);
    float4 x4 = *reinterpret_cast<const float4*>(A.vx + i0);
    float4 y4 = *reinterpret_cast<const float4*>(A.vy + i0);
    float4 z4 = *reinterpret_cast<const float4*>(A.vz + i0);
    ulonglong2 a = *reinterpret_cast<const ulonglong2*>(A.id + i0);
    ulonglong2 b = *reinterpret_cast<const ulonglong2*>(A.id + i0 + 2);
    c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
    f[0] = f4.x; f[1] = f4.y; f[2] = f4.z; f[3] = f4.w;
    vx[0] = x4.x; vx[1] = x4.y; vx[2] = x4.z; vx[3] = x4.w;
    vy[0] = y4.x; vy[1] = y4.y; vy[2] = y4.z; vy[3] = y4.w;
    vz[0] = z4.x; vz[1] = z4.y; vz[2] = z4.z; vz[3] = z4.w;
    id[0] = a.x; id[1] = a.y; id[2] = b.x; id[3] = b.y;
  } else {
#pragma unroll
    for (int k = 0; k < PIC_PPT; ++k) c[k] = PIC_DEAD_CELL;
  }
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  // claim the slots of all four particles first (four atomics in flight), then copy
  unsigned peers[PIC_PPT], base[PIC_PPT];
#pragma unroll
  for (int k = 0; k < PIC_PPT; ++k) {
    const bool live = c[k] != PIC_DEAD_CELL;
    const int cell = c[k] & PIC_CELL_MASK;  // the word also carries the null-collision countdown
    peers[k] = __match_any_sync(0xFFFFFFFFu, live ? cell : -1);
    base[k] = 0u;
    if (live && lane == __ffs(peers[k]) - 1) base[k] = atomicAdd(cur + cell, (unsigned)__popc(peers[k]));
  }
#pragma unroll
  for (int k = 0; k < PIC_PPT; ++k) {
    const unsigned b = __shfl_sync(0xFFFFFFFFu, base[k], __ffs(peers[k]) - 1);
    if (c[k] == PIC_DEAD_CELL) continue;
    const unsigned long long slot = b + (unsigned)__popc(peers[k] & below);
    if (slot >= P.cap[s]) {  // only reachable if the counts disagree with the arrays
      atomicOr(&P.ctl->error, ERR_DEVICE);
      continue;
    }
    D.cell[slot] = c[k];
    D.frac[slot] = f[k];
    D.vx[slot] = vx[k];
    D.vy[slot] = vy[k];
    D.vz[slot] = vz[k];
    D.id[slot] = id[k];
  }
}

__global__ void __launch_bounds__(PIC_TPB) k_sort_scatter(const SortParams P) {
  const unsigned long long n0 = P.ctl->sort_total[0], n1 = P.ctl->sort_total[1];
  const unsigned long long tiles0 = (n0 + PIC_TILE - 1) / PIC_TILE;
  const unsigned long long tiles = tiles0 + (n1 + PIC_TILE - 1) / PIC_TILE;
  for (unsigned long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    if (t < tiles0) {
      const unsigned long long i0 = t * PIC_TILE + (unsigned long long)threadIdx.x * PIC_PPT;
      scatter_tile<0>(P, i0, i0 < n0);
    } else {
      const unsigned long long i0 = (t - tiles0) * PIC_TILE + (unsigned long long)threadIdx.x * PIC_PPT;
      scatter_tile<1>(P, i0, i0 < n1);
    }
  }
}

void scan_attrs() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_sort_scan<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(unsigned int) * PIC_FIELD_SEG_MAX));
    cudaFuncSetAttribute(k_sort_scan<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(unsigned int) * PIC_FIELD_SEG_MAX));
    attr_set = true;
  }
}

}  // namespace

cudaError_t launch_sort_scan_batch(const SortParams* tab, int nsims, int maxN, cudaStream_t st) {
  if (nsims < 1 || nsims > PIC_BATCH_MAX || maxN < 2 || maxN > PIC_MAX_CELLS_FP32) return cudaErrorInvalidValue;
  scan_attrs();
  const int seg = (maxN + PIC_FIELD_CTAS - 1) / PIC_FIELD_CTAS;
  SortParams unused;
  memset(&unused, 0, sizeof(unused));
  k_sort_scan<true><<<2 * nsims * PIC_FIELD_CTAS, 1024, sizeof(unsigned int) * (size_t)seg, st>>>(unused, tab);
  return cudaGetLastError();
}

cudaError_t launch_sort32(Species32 src[2], Species32 dst[2], unsigned int* cnt[2],
                          unsigned int* cursor[2], const unsigned long long cap[2], Ctl* ctl, int N,
                          int grid, cudaStream_t st) {
  SortParams P;
  for (int s = 0; s < 2; ++s) {
    P.cap[s] = cap[s];
    P.src[s] = src[s];
    P.dst[s] = dst[s];
    P.cnt[s] = cnt[s];
    P.cursor[s] = cursor[s];
  }
  P.ctl = ctl;
  P.N = N;
  P.defer = 0;
  const int seg = (N + PIC_FIELD_CTAS - 1) / PIC_FIELD_CTAS;
  scan_attrs();
  k_sort_scan<false><<<2 * PIC_FIELD_CTAS, 1024, sizeof(unsigned int) * (size_t)seg, st>>>(P, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sort_scatter<<<grid, PIC_TPB, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_sort_scan32(Species32 src[2], Species32 dst[2], unsigned int* cnt[2], unsigned int* cursor[2],
                               const unsigned long long cap[2], Ctl* ctl, int N, cudaStream_t st) {
  SortParams P;
  for (int s = 0; s < 2; ++s) {
    P.cap[s] = cap[s];
    P.src[s] = src[s];
    P.dst[s] = dst[s];
    P.cnt[s] = cnt[s];
    P.cursor[s] = cursor[s];
  }
  P.ctl = ctl;
  P.N = N;
  P.defer = 1;
  const int seg = (N + PIC_FIELD_CTAS - 1) / PIC_FIELD_CTAS;
  scan_attrs();
  k_sort_scan<false><<<2 * PIC_FIELD_CTAS, 1024, sizeof(unsigned int) * (size_t)seg, st>>>(P, nullptr);
  return cudaGetLastError();
}
