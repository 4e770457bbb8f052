// k_field.cu -- deposit finalisation, field solve and node field of the PIC cycle (paper Sec. 2:
// "deposition to the grid" and "field solver"; BIT1's native Poisson solver).
//
// The interior problem -phi_{j-1} + 2 phi_j - phi_{j+1} = f_j = dx^2 rho_j (eps0 = 1),
// phi_0 = V_L, phi_N = V_R, has the exact inverse (discrete Green's function)
//   G_jk = min(j,k) (N - max(j,k)) / N,
//   phi_j = [ (N-j) A_j + j B_j ] / N + V_L (N-j)/N + V_R j/N,
//   A_j = sum_{k<=j} k f_k,  B_j = sum_{k>j} (N-k) f_k,
// and the node field is E_j = (phi_{j-1} - phi_{j+1}) / (2 dx) inside, Gauss's law over the half
// cell at the walls: E_0 = (phi_0 - phi_1)/dx - rho_0 dx/2, E_N = (phi_{N-1} - phi_N)/dx + rho_N dx/2.
//
// Two implementations, each one thread-block cluster of PIC_FIELD_CTAS CTAs; a CTA stages its
// contiguous segment of the N + 1 nodes in shared memory with coalesced loads, each thread scans a
// run of consecutive nodes, and CTA totals travel through distributed shared memory.  The CTA
// count is fixed, so every bit of the result is reproducible.
//
// k_field_exact (FP32 path, integer species charges; the per-step solve).  FP64 runs at a small
// fraction of the FP32/INT32 rate on this GPU, and the deposit is already exact int64, so the
// solve stays in integers: with r_j = m_0 R_0j + m_1 R_1j (m_s = q_s ppc_{1-s}, so that
// f_j = kappa r_j with kappa = dx^2 2^-32 / (ppc_0 ppc_1)), the cumulative charge Q_j = sum_{k<=j}
// r_k over interior nodes, and T = N Q_N - sum_k k r_k, the Green's-function formula reduces to
//   E_j = kappa / (2 N dx) * [ N (Q_j + Q_{j-1}) - 2 T ] + (V_L - V_R) / (N dx)       (0 < j < N)
//   E_0 = -kappa / (N dx) * [ T + N r_0 ] + (V_L - V_R) / (N dx),
//   E_N =  kappa / (N dx) * [ sum_k k r_k + N r_N ] + (V_L - V_R) / (N dx),
// (r_0, r_N: the wall-node deposits), with the brackets exact in int128 and one FP64 rounding per
// node.  phi and rho are needed only by the diagnostics and come from k_field_fp64 on demand.
//
// k_field_fp64 (plain FP64 path, the pic_poisson operation, diagnostics, non-integer charges):
// the Green's-function formula above in FP64 with two prefix scans.
//
// Density smoothing (Sec. 2, BIT1's smoothing operators): P.smooth passes of the binomial filter
// rho' = (rho_{j-1} + 2 rho_j + rho_{j+1}) / 4 inside, (rho_0 + rho_1) / 2 and
// (rho_{N-1} + rho_N) / 2 at the walls, applied to the charge before the solve.  In the exact
// kernel it runs on t_j = r_j dx / vol_j (the wall charges doubled) in integers, each pass the
// stencil times 4 (inside t_{j-1} + 2 t_j + t_{j+1}, at a wall 2 (t_0 + t_1)); r is then rebuilt in
// units of 2^-(2 passes + 1) of the deposit unit and the E coefficients carry that factor.  Each
// pass reads the neighbours of a thread's run of nodes (across CTAs through distributed shared
// memory), waits for the cluster, and rewrites the run in place.
#include <cooperative_groups.h>

#include <cstring>
#include <type_traits>

#include "pic_internal.cuh"

namespace cg = cooperative_groups;

namespace {

struct Pair {
  double a, c;
};

__device__ __forceinline__ Pair warp_incl_scan(Pair v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double a = __shfl_up_sync(0xFFFFFFFFu, v.a, o);
    double c = __shfl_up_sync(0xFFFFFFFFu, v.c, o);
    if (lane >= o) {
      v.a += a;
      v.c += c;
    }
  }
  return v;
}

__device__ __forceinline__ __int128 shfl_up_i128(__int128 v, int o) {
  long long lo = (long long)(unsigned long long)v;
  long long hi = (long long)(v >> 64);
  lo = __shfl_up_sync(0xFFFFFFFFu, lo, o);
  hi = __shfl_up_sync(0xFFFFFFFFu, hi, o);
  return ((__int128)hi << 64) | (__int128)(unsigned long long)lo;
}

__device__ __forceinline__ double i128_to_double(__int128 x) {
  const long long hi = (long long)(x >> 64);
  const unsigned long long lo = (unsigned long long)x;
  if ((hi == 0 && (long long)lo >= 0) || (hi == -1 && (long long)lo < 0)) return (double)(long long)lo;
  return (double)hi * 18446744073709551616.0 + (double)lo;
}

// node deposit R_sj from the per-cell counts and right-weight sums: R_j = 2^32 cnt_j - S_j + S_{j-1}
__device__ __forceinline__ long long node_R(const PoissonParams& P, int s, int j) {
  unsigned long long r = 0ull;
  if (j < P.N) r += ((unsigned long long)P.cnt[s][j] << 32) - P.S[s][j];
  if (j > 0) r += P.S[s][j - 1];
  return (long long)r;
}

// particle-array bookkeeping after the deposits of a step (one thread)
__device__ void bookkeeping(const PoissonParams& P) {
  Ctl* g = P.ctl;
  // after a scattering step the particles (and this step's births) are in the buffer the sort
  // scan sized: its extent is sort_new
  const unsigned long long c0 = P.scatter_step ? g->sort_new[0] : g->n_cur[0];
  const unsigned long long c1 = P.scatter_step ? g->sort_new[1] : g->n_cur[1];
  const unsigned long long b0 = g->n_born[0], b1 = g->n_born[1];
  const unsigned long long l0 = g->n_live[0], l1 = g->n_live[1], mark = g->live_mark;
  if (P.count_step) g->particle_steps += mark;
  g->live_mark = l0 + l1;
  for (int s = 0; s < 2; ++s) {
    unsigned long long n = (s ? c1 + b1 : c0 + b0);
    if (n > P.cap[s]) n = P.cap[s];
    const unsigned long long pad = round_up4(n);
    for (unsigned long long i = n; i < pad; ++i) {
      if (P.plain)
        P.pad64[s].x[i] = -1.0;
      else
        P.pad32[s].cell[i] = PIC_DEAD_CELL;
    }
    g->n_cur[s] = pad;
    g->n_born[s] = 0ull;
    g->ke_last[s] = g->ke_acc[s];
    g->ke_acc[s] = 0ull;
  }
  g->src_K = 0ull;
  g->wlog_n = 0ull;
  if (P.nt_cap && P.nt_pad.cell) {  // after a neutral step: the extent of the buffer it wrote
    unsigned long long n = (P.nt_append ? g->nt_cur : 0ull) + g->nt_out;
    if (n > P.nt_cap) n = P.nt_cap;
    const unsigned long long pad = round_up4(n);
    for (unsigned long long i = n; i < pad; ++i) P.nt_pad.cell[i] = PIC_DEAD_CELL;
    g->nt_cur = pad;
    g->nt_out = 0ull;
  }
}

// P.smooth passes of the density filter over this CTA's segment buf[0 .. len) of the nodes
// [a, a + len), in the thread-run layout (thread tid owns buf[i0 .. i0 + items)).  Long long: the
// integer stencil of the exact kernel on t (x 4 per pass); double: the filter on densities.
template <class T>
__device__ void smooth_segment(T* buf, int len, int a, int N, int seg, int i0, int items, int passes,
                               cg::cluster_group& cluster, int rank) {
  for (int pass = 0; pass < passes; ++pass) {
    cluster.sync();  // every CTA's segment holds the previous pass
    T left = T(0), right = T(0);
    if (i0 < len) {
      const int last = min(i0 + items, len) - 1;
      if (a + i0 > 0) left = i0 > 0 ? buf[i0 - 1] : cluster.map_shared_rank(buf, rank - 1)[seg - 1];
      if (a + last < N) right = last + 1 < len ? buf[last + 1] : cluster.map_shared_rank(buf, rank + 1)[0];
    }
    cluster.sync();  // every neighbour is read before any run is rewritten
    T prev = left;
    for (int k = 0; k < items; ++k) {
      const int i = i0 + k;
      if (i >= len) break;
      const int j = a + i;
      const T cur = buf[i];
      const T next = (k + 1 < items && i + 1 < len) ? buf[i + 1] : right;
      T v;
      if constexpr (std::is_integral<T>::value) {
        v = j == 0 ? T(2) * (cur + next) : (j == N ? T(2) * (prev + cur) : prev + T(2) * cur + next);
      } else {
        v = j == 0 ? (cur + next) * T(0.5) : (j == N ? (prev + cur) * T(0.5) : (prev + T(2) * cur + next) * T(0.25));
      }
      buf[i] = v;
      prev = cur;
    }
  }
}

// =============================================================================================
// BATCH: cluster k of the grid solves simulation k of an ensemble, with the parameters tab[k].
template <bool BATCH>
__global__ void __cluster_dims__(PIC_FIELD_CTAS, 1, 1) __launch_bounds__(PIC_FIELD_TPB, 1)
    k_field_exact(const __grid_constant__ PoissonParams P0, const PoissonParams* __restrict__ tab) {
  const PoissonParams& P = BATCH ? tab[blockIdx.x / PIC_FIELD_CTAS] : P0;
  extern __shared__ long long Rn[];  // r_j of this CTA's segment, then E_j (as double bits)
  __shared__ __int128 warp_q[PIC_FIELD_TPB / 32], warp_p[PIC_FIELD_TPB / 32];
  __shared__ __int128 cta_q, cta_p;  // read by the other CTAs of the cluster
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int TPB = (int)blockDim.x, nw = TPB >> 5;  // a multiple of 32, at most PIC_FIELD_TPB
  const int rank = (int)cluster.block_rank();
  const int N = P.N;
  const int M = N + 1;
  const int seg = (M + PIC_FIELD_CTAS - 1) / PIC_FIELD_CTAS;
  const int a = rank * seg;
  const int len = max(0, min(seg, M - a));

  if (P.ctl && !P.no_book && rank == 0 && tid == 0) bookkeeping(P);

  // ---- pass 1 (coalesced): node deposits, net integer charge ------------------------------------
  // |r| bound that keeps the smoothed values (at most 4^(passes + 1) |r|) inside int64
  const __int128 lim = (__int128)0x7FFFFFFFFFFFFFFFll >> (P.smooth ? 2 * P.smooth + 2 : 0);
  for (int i = tid; i < len; i += TPB) {
    const int j = a + i;
    // a decomposed simulation solves the total of every part's deposits (exact integer sums)
    const long long R0 = P.R_in ? P.R_in[j] : node_R(P, 0, j), R1 = P.R_in ? P.R_in[M + j] : node_R(P, 1, j);
    P.R[0][j] = R0;
    P.R[1][j] = R1;
    const __int128 rn = (__int128)P.m[0] * R0 + (__int128)P.m[1] * R1;
    if (rn > lim || rn < -lim) {
      atomicOr(&P.ctl->error, ERR_DEVICE);  // net deposit beyond int64: report, never wrap silently
    }
    Rn[i] = (long long)rn;
    if (P.NE2) {  // node electron density (neutral ionization)
      const float ne = (float)((double)R0 * P.ne_scale * ((j == 0 || j == N) ? 2.0 : 1.0));
      if (j < N) P.NE2[j].x = ne;
      if (j > 0) P.NE2[j - 1].y = ne;
    }
  }
  __syncthreads();

  const int items = (len + TPB - 1) / TPB;
  const int i0 = tid * items;
  if (P.smooth > 0) {
    for (int k = 0; k < items; ++k) {  // t: wall charges doubled
      const int i = i0 + k;
      if (i < len && (a + i == 0 || a + i == N)) Rn[i] *= 2;
    }
    smooth_segment<long long>(Rn, len, a, N, seg, i0, items, P.smooth, cluster, rank);
    for (int k = 0; k < items; ++k) {  // back to charges, in units of 2^-(2 passes + 1)
      const int i = i0 + k;
      if (i < len && a + i != 0 && a + i != N) Rn[i] *= 2;
    }
  }

  // ---- per-thread runs: Q (cumulative interior charge) and sum of k r_k -------------------------
  __int128 oq = 0, op = 0;
  for (int k = 0; k < items; ++k) {
    const int i = i0 + k;
    if (i >= len) break;
    const int j = a + i;
    if (j >= 1 && j <= N - 1) {
      oq += (__int128)Rn[i];
      op += (__int128)Rn[i] * j;
    }
  }
  __int128 iq = oq, ip = op;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const __int128 uq = shfl_up_i128(iq, o), up = shfl_up_i128(ip, o);
    if (lane >= o) {
      iq += uq;
      ip += up;
    }
  }
  if (lane == 31) {
    warp_q[w] = iq;
    warp_p[w] = ip;
  }
  __syncthreads();
  if (tid < 32) {
    __int128 vq = tid < nw ? warp_q[tid] : (__int128)0, vp = tid < nw ? warp_p[tid] : (__int128)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const __int128 uq = shfl_up_i128(vq, o), up = shfl_up_i128(vp, o);
      if (lane >= o) {
        vq += uq;
        vp += up;
      }
    }
    warp_q[tid] = vq;
    warp_p[tid] = vp;
    if (tid == 31) {
      cta_q = vq;
      cta_p = vp;
    }
  }
  __syncthreads();
  __int128 q = (w ? warp_q[w - 1] : (__int128)0) + iq - oq;  // exclusive prefix within the CTA
  cluster.sync();  // CTA totals visible; every input of pass 1 has been read
  __int128 Qtot = 0, Ptot = 0;
#pragma unroll
  for (int r = 0; r < PIC_FIELD_CTAS; ++r) {
    const __int128 vq = *cluster.map_shared_rank(&cta_q, r);
    const __int128 vp = *cluster.map_shared_rank(&cta_p, r);
    if (r < rank) q += vq;
    Qtot += vq;
    Ptot += vp;
  }
  // clear the deposit accumulators for the next step (coalesced)
  for (int i = tid; i < len; i += TPB) {
    const int j = a + i;
    if (j < N) {
      P.S[0][j] = 0ull;
      P.S[1][j] = 0ull;
      if (!P.keep_counts) {
        const_cast<unsigned int*>(P.cnt[0])[j] = 0u;
        const_cast<unsigned int*>(P.cnt[1])[j] = 0u;
      }
    }
  }

  // ---- pass 2: node field in place --------------------------------------------------------------
  const __int128 T = (__int128)N * Qtot - Ptot;
  for (int k = 0; k < items; ++k) {
    const int i = i0 + k;
    if (i >= len) break;
    const int j = a + i;
    const __int128 r = Rn[i];
    double E;
    if (j == 0) {
      E = -P.e_wall * i128_to_double(T + (__int128)N * r) + P.e_bias;
    } else if (j == N) {
      E = P.e_wall * i128_to_double(Ptot + (__int128)N * r) + P.e_bias;
    } else {
      const __int128 qprev = q;
      q += r;
      E = P.e_in * i128_to_double((__int128)N * (q + qprev) - 2 * T) + P.e_bias;
    }
    Rn[i] = __double_as_longlong(E);
  }
  __syncthreads();
  for (int i = tid; i < len; i += TPB) {
    const int j = a + i;
    const double E = __longlong_as_double(Rn[i]);
    P.E[j] = E;
    if (j < N) P.E2[j].x = (float)E;
    if (j > 0) P.E2[j - 1].y = (float)E;
  }
  cluster.sync();  // keep the shared totals alive until every CTA has read them
}

// =============================================================================================
// The same integer-exact solve over many CTAs (one simulation; k_field_exact's formulas and
// roundings, so the two give identical bits).  On one 8-CTA cluster the solve of a 65537-node
// grid is bound by the FP64 rate of eight SMs; here each of up to one CTA per SM takes a contiguous
// segment of nodes, and the CTAs exchange only their segment totals (interior charge and first
// moment) through global memory and one grid barrier.  The launch is cooperative, so every CTA is
// resident while the others wait.  Smoothing reads a halo of one node per pass on each side of
// the segment (recomputed from the deposits), so it needs no exchange.
constexpr int FG_TPB = 256;
constexpr size_t FG_SMEM_MAX = 96 * 1024;  // shared memory of one CTA: two buffers of its segment

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Sum of an int128 over the CTA (every thread gets it); red: FG_TPB / 32 entries of shared memory.
__device__ __forceinline__ __int128 block_sum_i128(__int128 v, __int128* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long lo = __shfl_xor_sync(0xFFFFFFFFu, (long long)(unsigned long long)v, o);
    const long long hi = __shfl_xor_sync(0xFFFFFFFFu, (long long)(v >> 64), o);
    v += ((__int128)hi << 64) | (__int128)(unsigned long long)lo;
  }
  __syncthreads();  // red is free
  if (lane == 0) red[w] = v;
  __syncthreads();
  __int128 t = 0;
#pragma unroll
  for (int k = 0; k < FG_TPB / 32; ++k) t += red[k];
  return t;
}

__global__ void __launch_bounds__(FG_TPB) k_field_grid(const __grid_constant__ PoissonParams P) {
  extern __shared__ long long fg[];  // two buffers of the extended segment (t, then E as bits)
  __shared__ __int128 warp_q[FG_TPB / 32], warp_p[FG_TPB / 32], red[FG_TPB / 32];
  __shared__ __int128 cta_q, cta_p;
  __shared__ int ok;
  FieldGrid* const G = P.grid;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  constexpr int nw = FG_TPB / 32;
  const int N = P.N, M = N + 1;
  const int nb = (int)gridDim.x, rank = (int)blockIdx.x;
  const int seg = (M + nb - 1) / nb;
  const int a = rank * seg;
  const int len = max(0, min(seg, M - a));
  const int h = P.smooth;                                  // halo: one node per pass
  const int xa = max(0, a - h), xb = min(M, a + len + h);  // extended segment [xa, xb)
  const int xl = max(0, xb - xa);
  long long* buf = fg;
  long long* alt = fg + (seg + 2 * h);

  if (P.ctl && !P.no_book && rank == 0 && tid == 0) bookkeeping(P);

  // ---- node deposits, net integer charge (own nodes stored, the halo only read) -------------------
  const __int128 lim = (__int128)0x7FFFFFFFFFFFFFFFll >> (h ? 2 * h + 2 : 0);
  for (int e = tid; e < xl; e += FG_TPB) {
    const int j = xa + e;
    const bool own = j >= a && j < a + len;
    const long long R0 = P.R_in ? P.R_in[j] : node_R(P, 0, j), R1 = P.R_in ? P.R_in[M + j] : node_R(P, 1, j);
    const __int128 rn = (__int128)P.m[0] * R0 + (__int128)P.m[1] * R1;
    if (own) {
      P.R[0][j] = R0;
      P.R[1][j] = R1;
      if (rn > lim || rn < -lim) atomicOr(&P.ctl->error, ERR_DEVICE);  // never wrap silently
      if (P.NE2) {
        const float ne = (float)((double)R0 * P.ne_scale * ((j == 0 || j == N) ? 2.0 : 1.0));
        if (j < N) P.NE2[j].x = ne;
        if (j > 0) P.NE2[j - 1].y = ne;
      }
    }
    buf[e] = (long long)rn;
  }
  __syncthreads();
  if (h > 0) {  // the integer filter of k_field_exact: t (wall charges doubled), x 4 per pass
    for (int e = tid; e < xl; e += FG_TPB) {
      const int j = xa + e;
      if (j == 0 || j == N) buf[e] *= 2;
    }
    __syncthreads();
    for (int pass = 0; pass < h; ++pass) {
      for (int e = tid; e < xl; e += FG_TPB) {
        const int j = xa + e;
        const long long cur = buf[e];
        long long v;
        if (j == 0)
          v = 2 * (cur + buf[e + 1]);
        else if (j == N)
          v = 2 * (buf[e - 1] + cur);
        else if (e == 0 || e == xl - 1)
          v = cur;  // the halo's edge: stale from here on, one node further each pass
        else
          v = buf[e - 1] + 2 * cur + buf[e + 1];
        alt[e] = v;
      }
      __syncthreads();
      long long* const t = buf;
      buf = alt;
      alt = t;
    }
    for (int e = tid; e < xl; e += FG_TPB) {  // back to charges, in units of 2^-(2 passes + 1)
      const int j = xa + e;
      if (j != 0 && j != N) buf[e] *= 2;
    }
    __syncthreads();
  }
  long long* const own_r = buf + (a - xa);

  // ---- per-thread runs of the own segment: Q (cumulative interior charge) and sum of k r_k -------
  const int items = (len + FG_TPB - 1) / FG_TPB;
  const int i0 = tid * items;
  __int128 oq = 0, op = 0;
  for (int k = 0; k < items; ++k) {
    const int i = i0 + k;
    if (i >= len) break;
    const int j = a + i;
    if (j >= 1 && j <= N - 1) {
      oq += (__int128)own_r[i];
      op += (__int128)own_r[i] * j;
    }
  }
  __int128 iq = oq, ip = op;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const __int128 uq = shfl_up_i128(iq, o), up = shfl_up_i128(ip, o);
    if (lane >= o) {
      iq += uq;
      ip += up;
    }
  }
  if (lane == 31) {
    warp_q[w] = iq;
    warp_p[w] = ip;
  }
  __syncthreads();
  if (tid < 32) {
    __int128 vq = tid < nw ? warp_q[tid] : (__int128)0, vp = tid < nw ? warp_p[tid] : (__int128)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const __int128 uq = shfl_up_i128(vq, o), up = shfl_up_i128(vp, o);
      if (lane >= o) {
        vq += uq;
        vp += up;
      }
    }
    if (tid < nw) {
      warp_q[tid] = vq;
      warp_p[tid] = vp;
    }
    if (tid == 31) {
      cta_q = vq;
      cta_p = vp;
    }
  }
  __syncthreads();
  __int128 q = (w ? warp_q[w - 1] : (__int128)0) + iq - oq;  // exclusive prefix within the CTA

  // ---- grid barrier: publish the CTA totals, wait for every CTA's ----------------------------------
  if (tid == 0) {
    G->tot[rank][0] = cta_q;
    G->tot[rank][1] = cta_p;
    const unsigned g0 = ld_acquire_u32(&G->gen);  // read before arriving: it cannot move until then
    __threadfence();
    int good = 1;
    if (atomicAdd(&G->count, 1u) == (unsigned)nb - 1u) {  // last to arrive: reset, release the rest
      G->count = 0u;
      __threadfence();
      atomicAdd(&G->gen, 1u);
    } else {
      good = 0;
      const unsigned long long t0 = global_ns();
      for (int it = 0; it < (1 << 22); ++it) {
        if (ld_acquire_u32(&G->gen) != g0) {
          good = 1;
          break;
        }
        if ((it & 63) == 63 && global_ns() - t0 > PIC_WAIT_LIMIT_NS) break;
      }
      if (!good) atomicOr(&P.ctl->error, ERR_TIMEOUT);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  if (!ok) return;  // reported; the field is left as it was

  // the prefix of the CTAs before this one and the grid totals (read past L1)
  __int128 pq = 0, tq = 0, tp = 0;
  for (int r = tid; r < nb; r += FG_TPB) {
    const long long* const t = reinterpret_cast<const long long*>(&G->tot[r][0]);
    const __int128 vq = ((__int128)__ldcg(t + 1) << 64) | (__int128)(unsigned long long)__ldcg(t);
    const __int128 vp = ((__int128)__ldcg(t + 3) << 64) | (__int128)(unsigned long long)__ldcg(t + 2);
    if (r < rank) pq += vq;
    tq += vq;
    tp += vp;
  }
  q += block_sum_i128(pq, red);
  const __int128 Qtot = block_sum_i128(tq, red);
  const __int128 Ptot = block_sum_i128(tp, red);

  // clear the deposit accumulators of the own segment for the next step (every CTA has read its
  // halo before the barrier)
  for (int i = tid; i < len; i += FG_TPB) {
    const int j = a + i;
    if (j < N) {
      P.S[0][j] = 0ull;
      P.S[1][j] = 0ull;
      if (!P.keep_counts) {
        const_cast<unsigned int*>(P.cnt[0])[j] = 0u;
        const_cast<unsigned int*>(P.cnt[1])[j] = 0u;
      }
    }
  }

  // ---- node field in place -------------------------------------------------------------------------
  const __int128 T = (__int128)N * Qtot - Ptot;
  for (int k = 0; k < items; ++k) {
    const int i = i0 + k;
    if (i >= len) break;
    const int j = a + i;
    const __int128 r = own_r[i];
    double E;
    if (j == 0) {
      E = -P.e_wall * i128_to_double(T + (__int128)N * r) + P.e_bias;
    } else if (j == N) {
      E = P.e_wall * i128_to_double(Ptot + (__int128)N * r) + P.e_bias;
    } else {
      const __int128 qprev = q;
      q += r;
      E = P.e_in * i128_to_double((__int128)N * (q + qprev) - 2 * T) + P.e_bias;
    }
    own_r[i] = __double_as_longlong(E);
  }
  __syncthreads();
  for (int i = tid; i < len; i += FG_TPB) {
    const int j = a + i;
    const double E = __longlong_as_double(own_r[i]);
    P.E[j] = E;
    if (j < N) P.E2[j].x = (float)E;
    if (j > 0) P.E2[j - 1].y = (float)E;
  }
}

// =============================================================================================
// FP64 Green's function.  MODE 0: from the per-cell counts (non-integer charges), 1: from the
// FP64 accumulators of the plain path, 2: from a given rho (pic_poisson), 3: from the stored R
// (diagnostics: rho and phi, and E only when asked for).
template <int MODE>
__device__ __forceinline__ double node_rho(const PoissonParams& P, int j) {
  const double inv_vol = (j == 0 || j == P.N) ? 2.0 * P.inv_dx : P.inv_dx;
  if (MODE == 0) {
    const long long R0 = node_R(P, 0, j), R1 = node_R(P, 1, j);
    P.R[0][j] = R0;
    P.R[1][j] = R1;
    return (P.qw[0] * (double)R0 + P.qw[1] * (double)R1) * 2.3283064365386963e-10 * inv_vol;
  } else if (MODE == 1) {
    const double a0 = P.acc[0][j], a1 = P.acc[1][j];
    P.R[0][j] = __double2ll_rn(a0 * 4294967296.0);
    P.R[1][j] = __double2ll_rn(a1 * 4294967296.0);
    return (P.qw[0] * a0 + P.qw[1] * a1) * inv_vol;
  } else if (MODE == 2) {
    return P.rho_in[j];
  } else {
    const long long R0 = P.R[0][j], R1 = P.R[1][j];
    if (P.zero_R) {  // each node is read by one thread
      P.R[0][j] = 0;
      P.R[1][j] = 0;
    }
    return (P.qw[0] * (double)R0 + P.qw[1] * (double)R1) * 2.3283064365386963e-10 * inv_vol;
  }
}

template <int MODE>
__global__ void __cluster_dims__(PIC_FIELD_CTAS, 1, 1) __launch_bounds__(PIC_FIELD_TPB, 1)
    k_field_fp64(const __grid_constant__ PoissonParams P) {
  extern __shared__ double F[];  // this CTA's segment: f_j = dx^2 rho_j, then phi_j
  __shared__ Pair warp_tot[PIC_FIELD_TPB / 32];
  __shared__ Pair cta_tot;  // read by the other CTAs of the cluster
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x;
  const int TPB = (int)blockDim.x, nw = TPB >> 5;  // a multiple of 32, at most PIC_FIELD_TPB
  const int rank = (int)cluster.block_rank();
  const int N = P.N;
  const int M = N + 1;
  const int seg = (M + PIC_FIELD_CTAS - 1) / PIC_FIELD_CTAS;
  const int a = rank * seg;
  const int len = max(0, min(seg, M - a));
  const double dx2 = P.dx * P.dx;

  if ((MODE == 0 || MODE == 1) && P.ctl && rank == 0 && tid == 0) bookkeeping(P);

  // ---- pass 1 (coalesced): node density -> shared f_j ---------------------------------------
  const int items = (len + TPB - 1) / TPB;
  const int i0 = tid * items;
  if (MODE == 3 && P.smooth > 0) {  // diagnostics of a smoothed run: the density the solve used
    for (int i = tid; i < len; i += TPB) F[i] = node_rho<MODE>(P, a + i);
    __syncthreads();
    smooth_segment<double>(F, len, a, N, seg, i0, items, P.smooth, cluster, rank);
    for (int k = 0; k < items; ++k) {
      const int i = i0 + k;
      if (i >= len) break;
      const int j = a + i;
      P.rho[j] = F[i];
      F[i] = (j >= 1 && j <= N - 1) ? dx2 * F[i] : 0.0;
    }
  } else {
    for (int i = tid; i < len; i += TPB) {
      const int j = a + i;
      const double r = node_rho<MODE>(P, j);
      if (MODE != 2) P.rho[j] = r;
      F[i] = (j >= 1 && j <= N - 1) ? dx2 * r : 0.0;
    }
  }
  __syncthreads();

  // ---- per-thread runs of consecutive nodes: sums of k f_k and (N - k) f_k ----------------------
  Pair own = {0.0, 0.0};
  for (int k = 0; k < items; ++k) {
    const int i = i0 + k;
    if (i >= len) break;
    const double f = F[i];
    const int j = a + i;
    own.a += (double)j * f;
    own.c += (double)(N - j) * f;
  }
  Pair incl = warp_incl_scan(own);
  if ((tid & 31) == 31) warp_tot[tid >> 5] = incl;
  __syncthreads();
  if (tid < 32) {
    Pair wi = warp_incl_scan(tid < nw ? warp_tot[tid] : Pair{0.0, 0.0});
    warp_tot[tid] = wi;  // inclusive over warps
    if (tid == 31) cta_tot = wi;
  }
  __syncthreads();
  Pair excl;
  {
    const int w = tid >> 5, lane = tid & 31;
    const double pa = __shfl_up_sync(0xFFFFFFFFu, incl.a, 1);
    const double pc = __shfl_up_sync(0xFFFFFFFFu, incl.c, 1);
    const Pair before = w ? warp_tot[w - 1] : Pair{0.0, 0.0};
    excl.a = before.a + (lane ? pa : 0.0);
    excl.c = before.c + (lane ? pc : 0.0);
  }
  cluster.sync();  // CTA totals visible; every input of pass 1 has been read
  Pair off = {0.0, 0.0}, tot = {0.0, 0.0};
#pragma unroll
  for (int r = 0; r < PIC_FIELD_CTAS; ++r) {
    const Pair v = *cluster.map_shared_rank(&cta_tot, r);
    if (r < rank) {
      off.a += v.a;
      off.c += v.c;
    }
    tot.a += v.a;
    tot.c += v.c;
  }
  // clear the accumulators of the deposit for the next step (coalesced)
  if (MODE == 0) {
    for (int i = tid; i < len; i += TPB) {
      const int j = a + i;
      if (j < N) {
        P.S[0][j] = 0ull;
        P.S[1][j] = 0ull;
        if (!P.keep_counts) {
          const_cast<unsigned int*>(P.cnt[0])[j] = 0u;
          const_cast<unsigned int*>(P.cnt[1])[j] = 0u;
        }
      }
    }
  } else if (MODE == 1) {
    for (int i = tid; i < len; i += TPB) {
      P.acc[0][a + i] = 0.0;
      P.acc[1][a + i] = 0.0;
    }
  }

  // ---- pass 2: potential, in place --------------------------------------------------------------
  double A = off.a + excl.a, Cc = off.c + excl.c;
  const double invN = 1.0 / (double)N;
  for (int k = 0; k < items; ++k) {
    const int i = i0 + k;
    if (i >= len) break;
    const int j = a + i;
    const double f = F[i];
    A += (double)j * f;
    Cc += (double)(N - j) * f;
    double phi;
    if (j == 0) {
      phi = P.V_L;
    } else if (j == N) {
      phi = P.V_R;
    } else {
      const double B = tot.c - Cc;
      phi = ((double)(N - j) * A + (double)j * B) * invN + P.V_L * ((double)(N - j) * invN) +
            P.V_R * ((double)j * invN);
    }
    F[i] = phi;
    P.phi[j] = phi;
  }
  cluster.sync();  // phi of the whole grid is written (shared here, global for the neighbours)

  // ---- pass 3 (coalesced): node field ------------------------------------------------------------
  if (P.E) {
    const double* rho = MODE == 2 ? P.rho_in : P.rho;
    for (int i = tid; i < len; i += TPB) {
      const int j = a + i;
      const double pm = j == 0 ? 0.0 : (i > 0 ? F[i - 1] : P.phi[j - 1]);
      const double pp = j == N ? 0.0 : (i + 1 < len ? F[i + 1] : P.phi[j + 1]);
      double E;
      if (j == 0)
        E = (F[i] - pp) * P.inv_dx - rho[0] * P.dx * 0.5;
      else if (j == N)
        E = (pm - F[i]) * P.inv_dx + rho[N] * P.dx * 0.5;
      else
        E = (pm - pp) * (0.5 * P.inv_dx);
      P.E[j] = E;
      if (P.E2) {
        if (j < N) P.E2[j].x = (float)E;
        if (j > 0) P.E2[j - 1].y = (float)E;
      }
    }
  }
  cluster.sync();  // keep the shared totals alive until every CTA has read them
}

template <class K>
void set_smem(K kernel, int bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

static void field_attrs() {
  static bool attr_set = false;
  if (!attr_set) {
    const int maxs = (int)(sizeof(double) * PIC_FIELD_SEG_MAX);
    set_smem(k_field_exact<false>, maxs);
    set_smem(k_field_exact<true>, maxs);
    set_smem(k_field_fp64<0>, maxs);
    set_smem(k_field_fp64<1>, maxs);
    set_smem(k_field_fp64<2>, maxs);
    set_smem(k_field_fp64<3>, maxs);
    attr_set = true;
  }
}

// Threads per CTA for a segment of seg nodes: about four nodes per thread (runs of consecutive
// nodes), a multiple of 32 between 64 and PIC_FIELD_TPB.  Small grids get small CTAs: the scans'
// FP64 and int128 work grows with the threads, not with the nodes.
static int field_tpb(int seg) {
  const int t = ((seg + 3) / 4 + 31) / 32 * 32;
  return t < 64 ? 64 : (t > PIC_FIELD_TPB ? PIC_FIELD_TPB : t);
}

cudaError_t launch_field(const PoissonParams& p, cudaStream_t st) {
  if (p.N < 2 || p.N > PIC_MAX_CELLS_FP32) return cudaErrorInvalidValue;
  const int seg = (p.N + 1 + PIC_FIELD_CTAS - 1) / PIC_FIELD_CTAS;
  const size_t smem = sizeof(double) * (size_t)seg;
  const int tpb = field_tpb(seg);
  field_attrs();
  switch (p.mode) {
    case 0:
      if (p.exact && p.grid && p.grid_ctas > 0) {
        const int nb = p.grid_ctas > PIC_FIELD_GRID_MAX ? PIC_FIELD_GRID_MAX : p.grid_ctas;
        const int gseg = (p.N + 1 + nb - 1) / nb;
        const size_t gsmem = sizeof(long long) * 2 * (size_t)(gseg + 2 * p.smooth);
        if (gsmem <= FG_SMEM_MAX) {  // else (very few SMs) the one-cluster solve below
          static bool grid_attr = false;
          if (!grid_attr) {
            set_smem(k_field_grid, (int)FG_SMEM_MAX);
            grid_attr = true;
          }
          void* args[] = {const_cast<PoissonParams*>(&p)};
          const cudaError_t e =
              cudaLaunchCooperativeKernel((const void*)k_field_grid, dim3(nb), dim3(FG_TPB), args, gsmem, st);
          if (e != cudaErrorCooperativeLaunchTooLarge) return e;
          cudaGetLastError();  // fewer SMs free than CTAs (a shared device): the one-cluster solve
        }
      }
      if (p.exact)
        k_field_exact<false><<<PIC_FIELD_CTAS, tpb, smem, st>>>(p, nullptr);
      else
        k_field_fp64<0><<<PIC_FIELD_CTAS, tpb, smem, st>>>(p);
      break;
    case 1: k_field_fp64<1><<<PIC_FIELD_CTAS, tpb, smem, st>>>(p); break;
    case 2: k_field_fp64<2><<<PIC_FIELD_CTAS, tpb, smem, st>>>(p); break;
    case 3: k_field_fp64<3><<<PIC_FIELD_CTAS, tpb, smem, st>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

namespace {
// This handle's node deposits R_sj = 2^32 cnt_j - S_j + S_{j-1} (the counts stay for the field
// kernel that closes the step).
__global__ void __launch_bounds__(256) k_node_deposit(const PoissonParams P, long long* __restrict__ out) {
  const int M = P.N + 1;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    out[j] = node_R(P, 0, j);
    out[M + j] = node_R(P, 1, j);
  }
}
}  // namespace

cudaError_t launch_node_deposit(const PoissonParams& p, long long* out, cudaStream_t st) {
  const int M = p.N + 1;
  const int grid = (M + 255) / 256 < 1024 ? (M + 255) / 256 : 1024;
  k_node_deposit<<<grid, 256, 0, st>>>(p, out);
  return cudaGetLastError();
}

// Integer-exact field of every simulation of an ensemble: one cluster per simulation, parameters
// tab[k] in device memory (their ctl, counts and arrays point into the batch's arrays).
cudaError_t launch_field_batch(const PoissonParams* tab, int nsims, int maxN, cudaStream_t st) {
  if (nsims < 1 || nsims > PIC_BATCH_MAX || maxN < 2 || maxN > PIC_MAX_CELLS_FP32) return cudaErrorInvalidValue;
  const int seg = (maxN + 1 + PIC_FIELD_CTAS - 1) / PIC_FIELD_CTAS;
  field_attrs();
  PoissonParams unused;
  memset(&unused, 0, sizeof(unused));
  k_field_exact<true><<<nsims * PIC_FIELD_CTAS, field_tpb(seg), sizeof(double) * (size_t)seg, st>>>(unused, tab);
  return cudaGetLastError();
}
