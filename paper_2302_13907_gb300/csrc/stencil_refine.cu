// Interface rows of the azimuthally refined grid (paper Sec. 3, "Azimuth grid
// refinement").  Each zone of the grid is a uniform grid with its own number
// of azimuthal nodes; where a stencil reaches across an interface it reads a
// ghost row holding the neighbouring zone's row at its own nodes.  Those rows
// are a linear map along theta of one row of the neighbour: the trigonometric
// (FFT zero-padding) interpolant coarse -> fine, and its adjoint fine ->
// coarse.  The maps are small dense matrices ([n_out][n_in], n <= 64) built on
// the host, so one launch after each half step applies all of them: block row
// = one transfer, thread = one z cell, the input column in registers, the
// matrix read as warp-uniform broadcasts.
#include "cwell_internal.cuh"

namespace cwell {
namespace {

constexpr int XF_THREADS = 128;

template <int NIN>
__device__ __forceinline__ void xfer_column(const XferDesc &d, int k) {
  float col[NIN];
#pragma unroll
  for (int ji = 0; ji < NIN; ji++) col[ji] = __ldg(d.src + ji * d.src_plane + k);
  for (int jo = 0; jo < d.n_out; jo++) {
    const float *m = d.mat + (long long)jo * NIN;
    float acc = 0.f;
#pragma unroll
    for (int ji = 0; ji < NIN; ji++) acc = fmaf(__ldg(m + ji), col[ji], acc);
    d.dst[jo * d.dst_plane + k] = acc;
  }
}

__global__ void __launch_bounds__(XF_THREADS) xfer_kernel(const __grid_constant__ XferParams p) {
  const XferDesc &d = p.d[blockIdx.y];
  const int k = blockIdx.x * XF_THREADS + threadIdx.x;
  if (k >= p.NZ) return;
  switch (d.n_in) {
    case 4: xfer_column<4>(d, k); break;
    case 8: xfer_column<8>(d, k); break;
    case 16: xfer_column<16>(d, k); break;
    case 32: xfer_column<32>(d, k); break;
    case 64: xfer_column<64>(d, k); break;
  }
}

}  // namespace

cudaError_t launch_xfer(const XferParams &p, cudaStream_t s) {
  if (p.n == 0) return cudaSuccess;  // one zone: no interface
  if (p.n < 0 || p.n > XFER_MAX || p.NZ < 1) return cudaErrorInvalidValue;
  for (int t = 0; t < p.n; t++) {
    const int n = p.d[t].n_in;
    if (n != 4 && n != 8 && n != 16 && n != 32 && n != 64) return cudaErrorInvalidValue;
  }
  xfer_kernel<<<dim3((p.NZ + XF_THREADS - 1) / XF_THREADS, p.n), XF_THREADS, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace cwell
