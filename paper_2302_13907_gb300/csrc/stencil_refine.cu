// Interface rows of the azimuthally refined grid (paper Sec. 3, "Azimuth grid
// refinement").  Each zone of the grid is a uniform grid with its own number
// of azimuthal nodes; where a stencil reaches across an interface it reads a
// ghost row holding the neighbouring zone's row at its own nodes.  Those rows
// are a linear map along theta of one row of the neighbour: the trigonometric
// (FFT zero-padding) interpolant coarse -> fine, and its adjoint fine ->
// coarse.  The maps are small dense matrices ([n_out][n_in], n <= 64) built on
// the host, so one launch after each half step applies all of them: block row
// = one transfer, block layer = XF_OUT consecutive outputs, thread = one z
// cell; the input column in registers, XF_OUT independent accumulations, the
// matrix read as warp-uniform broadcasts.
#include <algorithm>

#include "cwell_internal.cuh"

namespace cwell {
namespace {

constexpr int XF_THREADS = 128;
constexpr int XF_OUT = 4;  // outputs per block (every n_out is a multiple of 4)

template <int NIN>
__device__ __forceinline__ void xfer_column(const XferDesc &d, int jo0, int k) {
  float col[NIN];
#pragma unroll
  for (int ji = 0; ji < NIN; ji++) col[ji] = __ldg(d.src + ji * d.src_plane + k);
  float acc[XF_OUT];
#pragma unroll
  for (int o = 0; o < XF_OUT; o++) acc[o] = 0.f;
#pragma unroll
  for (int ji = 0; ji < NIN; ji++)
#pragma unroll
    for (int o = 0; o < XF_OUT; o++) acc[o] = fmaf(__ldg(d.mat + (long long)(jo0 + o) * NIN + ji), col[ji], acc[o]);
#pragma unroll
  for (int o = 0; o < XF_OUT; o++) d.dst[(jo0 + o) * d.dst_plane + k] = acc[o];
}

__global__ void __launch_bounds__(XF_THREADS) xfer_kernel(const __grid_constant__ XferParams p) {
  const XferDesc &d = p.d[blockIdx.y];
  const int k = blockIdx.x * XF_THREADS + threadIdx.x, jo0 = blockIdx.z * XF_OUT;
  if (k >= p.NZ || jo0 >= d.n_out) return;
  switch (d.n_in) {
    case 4: xfer_column<4>(d, jo0, k); break;
    case 8: xfer_column<8>(d, jo0, k); break;
    case 16: xfer_column<16>(d, jo0, k); break;
    case 32: xfer_column<32>(d, jo0, k); break;
    case 64: xfer_column<64>(d, jo0, k); break;
  }
}

}  // namespace

cudaError_t launch_xfer(const XferParams &p, cudaStream_t s) {
  if (p.n == 0) return cudaSuccess;  // one zone: no interface
  if (p.n < 0 || p.n > XFER_MAX || p.NZ < 1) return cudaErrorInvalidValue;
  int nz_out = 1;
  for (int t = 0; t < p.n; t++) {
    const int n = p.d[t].n_in, o = p.d[t].n_out;
    if (n != 4 && n != 8 && n != 16 && n != 32 && n != 64) return cudaErrorInvalidValue;
    if (o < XF_OUT || o % XF_OUT) return cudaErrorInvalidValue;
    nz_out = std::max(nz_out, o / XF_OUT);
  }
  xfer_kernel<<<dim3((p.NZ + XF_THREADS - 1) / XF_THREADS, p.n, nz_out), XF_THREADS, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace cwell
