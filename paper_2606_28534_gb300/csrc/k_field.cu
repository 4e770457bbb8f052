// k_field.cu -- deposit finalisation, field solve and node field of the PIC cycle (paper Sec. 2:
// "deposition to the grid" and "field solver"; BIT1's native Poisson solver).
//
// One thread-block cluster of PIC_FIELD_CTAS CTAs handles the whole grid (N + 1 nodes; each
// thread a run of consecutive nodes):
//   1. node deposits R_sj from the per-cell counts and right-weight sums written by the particle
//      step (R_j = 2^32 cnt_j - S_j + S_{j-1}, exact int64), node density
//      rho_j = sum_s q_s w_s R_sj 2^-32 / vol_j (vol = dx inside, dx/2 at the walls);
//   2. the interior problem -phi_{j-1} + 2 phi_j - phi_{j+1} = f_j = dx^2 rho_j (eps0 = 1),
//      phi_0 = V_L, phi_N = V_R, solved by its exact inverse (the discrete Green's function
//      G_jk = min(j,k) (N - max(j,k)) / N):
//        phi_j = [ (N-j) A_j + j B_j ] / N + V_L (N-j)/N + V_R j/N,
//        A_j = sum_{k<=j} k f_k,   B_j = sum_{k>j} (N-k) f_k,
//      i.e. two FP64 prefix scans; the CTA totals are exchanged through distributed shared memory;
//   3. E_j = (phi_{j-1} - phi_{j+1}) / (2 dx) inside, Gauss's law over the half cell at the
//      walls, stored as FP64 and as the node pairs (E_c, E_{c+1}) in FP32 that the particles read.
// The CTA count is fixed, so the summation order, and hence every bit of phi, is reproducible.
#include <cooperative_groups.h>

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

template <int MODE>
__device__ __forceinline__ double node_rho(const PoissonParams& P, int j) {
  const int N = P.N;
  const double vol = (j == 0 || j == N) ? 0.5 * P.dx : P.dx;
  if (MODE == 0) {
    long long R[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      unsigned long long r = 0ull;
      if (j < N) r += ((unsigned long long)P.cnt[s][j] << 32) - P.S[s][j];
      if (j > 0) r += P.S[s][j - 1];
      R[s] = (long long)r;
      P.R[s][j] = R[s];
    }
    return (P.qw[0] * (double)R[0] + P.qw[1] * (double)R[1]) * 2.3283064365386963e-10 / vol;
  } else if (MODE == 1) {
    double a0 = P.acc[0][j], a1 = P.acc[1][j];
    P.R[0][j] = __double2ll_rn(a0 * 4294967296.0);
    P.R[1][j] = __double2ll_rn(a1 * 4294967296.0);
    return (P.qw[0] * a0 + P.qw[1] * a1) / vol;
  } else {
    return P.rho_in[j];
  }
}

template <int MODE>
__global__ void __cluster_dims__(PIC_FIELD_CTAS, 1, 1) __launch_bounds__(PIC_FIELD_TPB, 1)
    k_field(const PoissonParams P) {
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ Pair warp_tot[PIC_FIELD_TPB / 32];
  __shared__ Pair cta_tot;  // read by the other CTAs of the cluster
  const int tid = threadIdx.x;
  const int rank = (int)cluster.block_rank();
  const int N = P.N;
  const int M = N + 1;
  const int items = (M + PIC_FIELD_CTAS * PIC_FIELD_TPB - 1) / (PIC_FIELD_CTAS * PIC_FIELD_TPB);
  const int j0 = (rank * PIC_FIELD_TPB + tid) * items;
  const double dx2 = P.dx * P.dx;

  // ---- pass 1: density, and per-thread sums of k f_k and (N - k) f_k ---------------------------
  Pair own = {0.0, 0.0};
  for (int k = 0; k < items; ++k) {
    const int j = j0 + k;
    if (j > N) break;
    double r = node_rho<MODE>(P, j);
    if (MODE != 2) P.rho[j] = r;
    if (j >= 1 && j <= N - 1) {
      double f = dx2 * r;
      own.a += (double)j * f;
      own.c += (double)(N - j) * f;
    }
  }
  // ---- block scan, then cluster scan of the CTA totals ------------------------------------------
  Pair incl = warp_incl_scan(own);
  if ((tid & 31) == 31) warp_tot[tid >> 5] = incl;
  __syncthreads();
  if (tid < 32) {
    Pair w = warp_tot[tid];
    Pair wi = warp_incl_scan(w);
    warp_tot[tid] = wi;  // inclusive over warps
    if (tid == 31) cta_tot = wi;
  }
  __syncthreads();
  Pair excl;  // exclusive prefix of this thread within the CTA
  {
    const int w = tid >> 5, lane = tid & 31;
    double pa = __shfl_up_sync(0xFFFFFFFFu, incl.a, 1);
    double pc = __shfl_up_sync(0xFFFFFFFFu, incl.c, 1);
    Pair before = w ? warp_tot[w - 1] : Pair{0.0, 0.0};
    excl.a = before.a + (lane ? pa : 0.0);
    excl.c = before.c + (lane ? pc : 0.0);
  }
  cluster.sync();
  Pair off = {0.0, 0.0}, tot = {0.0, 0.0};
  for (int r = 0; r < PIC_FIELD_CTAS; ++r) {
    const Pair* t = cluster.map_shared_rank(&cta_tot, r);
    Pair v = *t;
    if (r < rank) {
      off.a += v.a;
      off.c += v.c;
    }
    tot.a += v.a;
    tot.c += v.c;
  }
  // inputs are consumed: clear the accumulators for the next step
  for (int k = 0; k < items; ++k) {
    const int j = j0 + k;
    if (j > N) break;
    if (MODE == 0 && j < N) {
      P.S[0][j] = 0ull;
      P.S[1][j] = 0ull;
      if (!P.keep_counts) {
        const_cast<unsigned int*>(P.cnt[0])[j] = 0u;
        const_cast<unsigned int*>(P.cnt[1])[j] = 0u;
      }
    } else if (MODE == 1) {
      P.acc[0][j] = 0.0;
      P.acc[1][j] = 0.0;
    }
  }

  // ---- pass 2: potential --------------------------------------------------------------------
  double A = off.a + excl.a, Cc = off.c + excl.c;
  const double invN = 1.0 / (double)N;
  for (int k = 0; k < items; ++k) {
    const int j = j0 + k;
    if (j > N) break;
    if (j >= 1 && j <= N - 1) {
      double r = MODE == 2 ? P.rho_in[j] : P.rho[j];
      double f = dx2 * r;
      A += (double)j * f;
      Cc += (double)(N - j) * f;
    }
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
    P.phi[j] = phi;
  }
  cluster.sync();  // phi of the whole grid is visible to every CTA of the cluster

  // ---- pass 3: node field -----------------------------------------------------------------------
  const double* phi = P.phi;
  const double* rho = MODE == 2 ? P.rho_in : P.rho;
  for (int k = 0; k <= items; ++k) {
    const int j = j0 + k;
    if (j > N) break;
    double E;
    if (j == 0)
      E = (phi[0] - phi[1]) / P.dx - rho[0] * P.dx * 0.5;
    else if (j == N)
      E = (phi[N - 1] - phi[N]) / P.dx + rho[N] * P.dx * 0.5;
    else
      E = (phi[j - 1] - phi[j + 1]) / (2.0 * P.dx);
    if (k < items) P.E[j] = E;
    if (P.E2) {
      // node pair of cell j (left node) and of cell j-1 (right node)
      if (k < items && j < N) P.E2[j].x = (float)E;
      if (k > 0 && j >= 1) P.E2[j - 1].y = (float)E;
    }
  }

  // ---- bookkeeping of the particle arrays (one thread) ------------------------------------------
  if (P.ctl && rank == 0 && tid == 0) {
    Ctl* g = P.ctl;
    if (P.count_step) g->particle_steps += g->live_mark;
    g->live_mark = g->n_live[0] + g->n_live[1];
    for (int s = 0; s < 2; ++s) {
      unsigned long long n = g->n_cur[s] + g->n_born[s];
      if (n > P.cap[s]) n = P.cap[s];
      unsigned long long pad = round_up4(n);
      for (unsigned long long i = n; i < pad; ++i) {
        if (P.plain)
          P.pad64[s].x[i] = -1.0;
        else
          P.pad32[s].cell[i] = PIC_DEAD_CELL;
      }
      g->n_cur[s] = pad;
      g->n_born[s] = 0ull;
    }
    g->src_K = 0ull;
  }
}

}  // namespace

cudaError_t launch_field(const PoissonParams& p, cudaStream_t st) {
  if (p.N < 2 || p.N > PIC_MAX_CELLS_FP32) return cudaErrorInvalidValue;
  if (p.mode == 0)
    k_field<0><<<PIC_FIELD_CTAS, PIC_FIELD_TPB, 0, st>>>(p);
  else if (p.mode == 1)
    k_field<1><<<PIC_FIELD_CTAS, PIC_FIELD_TPB, 0, st>>>(p);
  else
    k_field<2><<<PIC_FIELD_CTAS, PIC_FIELD_TPB, 0, st>>>(p);
  return cudaGetLastError();
}
