// Device watchdog of a simulator handle (opts.watchdog_every = K > 0).
//
// After every K-th step an energy proxy of the whole state is summed on the
// device,
//     E = 1/2 sum over owned cells [ rho (v_r^2 + v_phi^2 + v_z^2)
//         + (s_rr^2 + s_phiphi^2 + s_zz^2 + 2 (s_rphi^2 + s_phiz^2 + s_rz^2)) / M ],
// rho and M = lambda + 2 mu (the P-wave modulus) of the cell's material, all
// values in physical units (the storage scales undone), every staggered
// component taken at its cell.  Kinetic energy is exact; the stress term is
// within a factor of about 0.3 to 3 of the elastic strain energy for any
// isotropic material, so E tracks the energy of Eq. 1 up to that factor.
// Once the source has stopped injecting (the last step of its wavelet table)
// the energy of the damped system cannot grow, so the first proxy taken
// after that is the reference, and the watchdog trips when a later proxy is
// more than WATCH_GROWTH times the reference, or when any proxy is not
// finite (a NaN or infinity anywhere in the fields).  A trip sets bit 3 of the
// handle's status word; sim_sync then returns SIM_EUNSTABLE.
//
// Both launches read the device step counter and return at once on the
// other steps, so they can sit in every captured step of a graph.
#include "cwell_internal.cuh"

namespace cwell {
namespace {

constexpr int WATCH_THREADS = 256;

__device__ __forceinline__ double sq(double x) { return x * x; }

template <typename T>
__device__ __forceinline__ double ld(const void *f, long long c) {
  return (double)St<T>::ld1((const T *)f + c);
}

template <typename T>
__global__ void __launch_bounds__(WATCH_THREADS) watch_reduce(const WParams p) {
  const int n = *p.step;
  if (n % p.every != 0) return;  // the same for every block
  const long long rows = (long long)p.nth * p.NR;
  double acc = 0.0;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const long long c0 = row * p.NZp;
    for (int k = p.k_lo + threadIdx.x; k < p.k_hi; k += WATCH_THREADS) {
      const long long c = c0 + k;
      const int m = p.id[c];
      const float rho = p.m_rho[m], M = p.m_lam[m].y;
      // squares in FP64: a growing (unstable) state stays finite here long after
      // its squares would overflow FP32
      const double v2 = sq(ld<T>(p.f[F_VR], c)) + sq(ld<T>(p.f[F_VP], c)) + sq(ld<T>(p.f[F_VZ], c));
      const double s2 = sq(ld<T>(p.f[F_SRR], c)) + sq(ld<T>(p.f[F_SPP], c)) + sq(ld<T>(p.f[F_SZZ], c)) +
                        2.0 * (sq(ld<T>(p.f[F_SRP], c)) + sq(ld<T>(p.f[F_SPZ], c)) + sq(ld<T>(p.f[F_SRZ], c)));
      acc += 0.5 * ((double)rho * v2 * p.iv2 + (M > 0.f ? s2 / (double)M * p.is2 : 0.0));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[WATCH_THREADS / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < WATCH_THREADS / 32; w++) s += part[w];
    atomicAdd(p.acc, s);
  }
}

// one thread: the decision on the sum the reduction left in acc[0]
__global__ void watch_check(const WParams p) {
  const int n = *p.step;
  if (n % p.every != 0) return;
  double *a = p.acc;
  const double E = a[0];
  a[0] = 0.0;
  a[1] = E;
  a[3] = (double)n;
  if (!isfinite(E)) {
    atomicOr(p.status, 8);
    return;
  }
  if (n < p.n_quiet) return;
  if (!(a[2] > 0.0)) {
    a[2] = E;  // the reference: the first proxy once the source is silent
    return;
  }
  if (E > WATCH_GROWTH * a[2]) atomicOr(p.status, 8);
}

}  // namespace

cudaError_t launch_watchdog(int storage, const WParams &p, int blocks, cudaStream_t s) {
  if (p.every <= 0) return cudaSuccess;
  switch (storage) {
    case 0: watch_reduce<float><<<blocks, WATCH_THREADS, 0, s>>>(p); break;
    case 1: watch_reduce<__nv_bfloat16><<<blocks, WATCH_THREADS, 0, s>>>(p); break;
    case 2: watch_reduce<__half><<<blocks, WATCH_THREADS, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  watch_check<<<1, 1, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace cwell
