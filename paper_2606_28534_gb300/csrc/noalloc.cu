// noalloc.cu -- pic_field_noalloc: the deposit and field solve of a caller's particle state with
// no device allocation at all.
//
// Who needs this: callers that cannot call cudaMalloc or go through an allocator, e.g. code that
// runs inside another framework's memory pool with a fixed budget, code that must not allocate
// after start-up (allocation can synchronise the device or fail late), or a host that hands over
// only its own input and output buffers.  Every other entry point of this library takes its
// device memory from the caller's workspace or allocates it; this one keeps the little scratch it
// needs (per-cell counts and right-weight sums, the FP32 node pairs and an error word) in a
// file-scope __device__ array of fixed size, which every GPU that loads the library holds until
// the process exits.
//
// It is a variant of the deposit half of the step kernel (CIC in int64 fixed point:
// W_r = rint(f 2^32), per-cell count and sum of W_r) followed by the integer-exact field kernel.
// Calls share the one scratch array: each call clears what must start at zero, and calls that
// overlap on the GPU (two streams, or two host threads) race on it.
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace {

constexpr int kMaxCells = PIC_NOALLOC_MAX_CELLS;
constexpr size_t kCtlBytes = (sizeof(Ctl) + 255) & ~size_t(255);
constexpr size_t kCntOff = kCtlBytes;                                      // u32 cnt[2][max]
constexpr size_t kSOff = kCntOff + 2 * sizeof(unsigned int) * kMaxCells;   // u64 S[2][max]
constexpr size_t kE2Off = kSOff + 2 * sizeof(unsigned long long) * kMaxCells;  // float2 E2[max]
constexpr size_t kScratchBytes = kE2Off + sizeof(float2) * kMaxCells;

// The scratch.  In host code this name is only a stand-in for the device symbol: its device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (set-up on the first call per device).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIC_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return PIC_ECUDA;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return PIC_OK;
}

// Deposit of the particles of one species into the per-cell scratch.  Particles with a cell
// outside [0, N) or a fraction outside [0, 1) are left out.
__global__ void __launch_bounds__(256) k_deposit_noalloc(const int* __restrict__ cell, const float* __restrict__ frac,
                                                         unsigned long long n, int N, unsigned int* __restrict__ cnt,
                                                         unsigned long long* __restrict__ S) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int c = cell[i];
    const float f = frac[i];
    if ((unsigned)c >= (unsigned)N || !(f >= 0.f && f < 1.f)) continue;
    atomicAdd(cnt + c, 1u);
    atomicAdd(S + c, (unsigned long long)__float2uint_rn(f * 4294967296.0f));
  }
}

}  // namespace

extern "C" int pic_field_noalloc(const pic_config* cfg, const int32_t* cell0, const float* frac0, uint64_t n0,
                                 const int32_t* cell1, const float* frac1, uint64_t n1, int64_t* R, double* E,
                                 void* cuda_stream) {
  if (!cfg || cfg->abi_version != PIC_ABI_VERSION || !R || !E) return PIC_EINVAL;
  if (cfg->ncells < 2 || cfg->ncells > kMaxCells) return PIC_EINVAL;  // beyond the fixed scratch
  if (!(cfg->L > 0) || cfg->ppc[0] < 1 || cfg->ppc[1] < 1) return PIC_EINVAL;
  if ((n0 && (!cell0 || !frac0)) || (n1 && (!cell1 || !frac1))) return PIC_EINVAL;
  if (cfg->smooth_passes < 0 || cfg->smooth_passes > PIC_MAX_SMOOTH) return PIC_EINVAL;
  // integer-exact field only: small integer charges, as in the step's own solve
  PoissonParams F;
  std::memset(&F, 0, sizeof(F));
  const long long g = std::gcd((long long)cfg->ppc[0], (long long)cfg->ppc[1]);
  for (int s = 0; s < 2; ++s) {
    const double q = cfg->charge[s];
    const long long other = (long long)cfg->ppc[1 - s] / g;
    if (q == 0.0 || q != std::floor(q) || std::fabs(q) > 64.0 || other > 1024) return PIC_EINVAL;
    F.m[s] = (long long)q * other;
  }
  const int N = cfg->ncells;
  const double dx = cfg->L / N;
  const double kappa = dx * dx * 2.3283064365386963e-10 * (double)g / ((double)cfg->ppc[0] * (double)cfg->ppc[1]);
  // smoothing leaves the net charge in units of 2^-(2 passes + 1) of the deposit unit, as in the
  // step's own solve
  const double unit = cfg->smooth_passes > 0 ? std::ldexp(1.0, -(2 * cfg->smooth_passes + 1)) : 1.0;
  F.e_in = unit * kappa / (2.0 * N * dx);
  F.e_wall = unit * kappa / ((double)N * dx);
  F.smooth = cfg->smooth_passes;
  F.e_bias = (cfg->V_left - cfg->V_right) / ((double)N * dx);
  F.exact = 1;
  F.mode = 0;
  F.N = N;
  F.dx = dx;
  F.inv_dx = 1.0 / dx;
  F.V_L = cfg->V_left;
  F.V_R = cfg->V_right;

  void* base = nullptr;
  const int rc = scratch_address(&base);
  if (rc != PIC_OK) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  Ctl* ctl = reinterpret_cast<Ctl*>(b);
  unsigned int* cnt[2] = {reinterpret_cast<unsigned int*>(b + kCntOff),
                          reinterpret_cast<unsigned int*>(b + kCntOff) + kMaxCells};
  unsigned long long* S[2] = {reinterpret_cast<unsigned long long*>(b + kSOff),
                              reinterpret_cast<unsigned long long*>(b + kSOff) + kMaxCells};
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the previous call's contents stay in the array: clear what the deposit accumulates into
  if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), st) != cudaSuccess) return PIC_ECUDA;
  for (int s = 0; s < 2; ++s) {
    if (cudaMemsetAsync(cnt[s], 0, sizeof(unsigned int) * N, st) != cudaSuccess ||
        cudaMemsetAsync(S[s], 0, sizeof(unsigned long long) * N, st) != cudaSuccess)
      return PIC_ECUDA;
  }
  const int32_t* cells[2] = {cell0, cell1};
  const float* fracs[2] = {frac0, frac1};
  const uint64_t ns[2] = {n0, n1};
  for (int s = 0; s < 2; ++s) {
    if (!ns[s]) continue;
    const unsigned long long blocks = (ns[s] + 255) / 256;
    const int grid = (int)(blocks < 152ull * 8 ? blocks : 152ull * 8);
    k_deposit_noalloc<<<grid, 256, 0, st>>>(cells[s], fracs[s], ns[s], N, cnt[s], S[s]);
    if (cudaGetLastError() != cudaSuccess) return PIC_ECUDA;
  }
  for (int s = 0; s < 2; ++s) {
    F.cnt[s] = cnt[s];
    F.S[s] = S[s];
  }
  F.R[0] = reinterpret_cast<long long*>(R);
  F.R[1] = reinterpret_cast<long long*>(R) + (N + 1);
  F.E = E;
  F.E2 = reinterpret_cast<float2*>(b + kE2Off);
  F.ctl = ctl;  // with zero capacities its particle bookkeeping touches no array
  if (launch_field(F, st) != cudaSuccess) return PIC_ECUDA;
  unsigned int err = 0;
  if (cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpy(&err, &ctl->error, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PIC_ECUDA;
  return err ? PIC_EDEVICE : PIC_OK;
}
