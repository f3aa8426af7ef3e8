// Trace surrogate: a small MLP + transposed-convolution decoder trained and
// run with hand-written kernels.
//
//   h1 = gelu(x W1 + b1)                      6 -> H1
//   h2 = gelu(h1 W2 + b2)                     H1 -> H2
//   a0 = gelu(reshape(h2 W3 + b3, [L0, C0]))  channels last
//   a_{l+1} = gelu(convT(a_l; T_l, t_l))      kernel 4, stride 2, padding 1
//   y = a_5 Wf + bf                           1x1 convolution to 8 receivers
//
// Every contraction is a GEMM on the tensor cores (BF16 operands, FP32
// accumulation): dense layers directly; a transposed convolution as
// Z = a T (T viewed as [C_in][C_out*4]) followed by a col2im sum of the two
// taps landing on each output position; its backward as im2col + two GEMMs.
// Weights are kept as FP32 masters (Adam) with BF16 copies for the GEMMs;
// activations are BF16 at every GEMM input, FP32 elsewhere.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/cwell.h"
#include "cwell_internal.cuh"

namespace cwell {

// ------------------------------------------------------------------ GEMM
// C[M x N] = alpha * op(A)[M x K] * op(B)[K x N] + beta * C, A and B BF16
// row-major (op = transpose when TA / TB), C FP32 row-major.  64 x 64 tiles,
// K step 32, four warps of 32 x 32, mma.sync m16n8k16 (BF16 in, FP32 acc).
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) gemm_bf16(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda,
                                                 const __nv_bfloat16 *__restrict__ B, int ldb, float *__restrict__ C,
                                                 int ldc, float alpha, float beta) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + GPAD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4][4] = {};
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < K; k0 += GBK) {
    // stage op(A)[m0.., k0..] as As[m][k] and op(B)[k0.., n0..] as Bs[n][k]
    for (int q = tid; q < GBM * GBK; q += 128) {
      const int mm = TA ? q % GBM : q / GBK, kk = TA ? q / GBM : q % GBK;
      const int m = m0 + mm, k = k0 + kk;
      As[mm][kk] = (m < M && k < K) ? (TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : zero;
    }
    for (int q = tid; q < GBN * GBK; q += 128) {
      const int nn = TB ? q / GBK : q % GBN, kk = TB ? q % GBK : q / GBN;
      const int n = n0 + nn, k = k0 + kk;
      Bs[nn][kk] = (n < N && k < K) ? (TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]) : zero;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; i++) {
        const int r = wm + 16 * i + g;
        af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 2 * t]);
        af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 2 * t]);
        af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 2 * t + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int c = wn + 8 * j + g;
        bfr[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][ks + 2 * t]);
        bfr[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int m = m0 + wm + 16 * i + g + (e >= 2 ? 8 : 0);
        const int n = n0 + wn + 8 * j + 2 * t + (e & 1);
        if (m < M && n < N) {
          float *cp = C + (long long)m * ldc + n;
          *cp = alpha * acc[i][j][e] + (beta != 0.f ? beta * *cp : 0.f);
        }
      }
}

static cudaError_t gemm_mma(bool ta, bool tb, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                            const __nv_bfloat16 *B, int ldb, float *C, int ldc, float alpha, float beta,
                            cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grd((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  if (!ta && !tb) gemm_bf16<false, false><<<grd, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
  else if (!ta && tb) gemm_bf16<false, true><<<grd, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
  else if (ta && !tb) gemm_bf16<true, false><<<grd, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
  else gemm_bf16<true, true><<<grd, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
  return cudaGetLastError();
}

// Path of a GEMM: products with at least 128 rows run on the tcgen05 kernel
// (gemm_tc.cu: 128 x 128 tiles, accumulator in tensor memory); the narrow
// ones (weight gradients: rows = channels) on the mma.sync kernel above.
// path: 0 = by shape, 1 = mma.sync, 2 = tcgen05.
static cudaError_t gemm_path(int path, bool ta, bool tb, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                             const __nv_bfloat16 *B, int ldb, float *C, int ldc, float alpha, float beta,
                             cudaStream_t s) {
  const bool tc = path == 2 || (path == 0 && M >= 128);
  return tc ? gemm_tcgen05(ta, tb, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, s)
            : gemm_mma(ta, tb, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, s);
}

static cudaError_t gemm(bool ta, bool tb, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                        const __nv_bfloat16 *B, int ldb, float *C, int ldc, float alpha, float beta, cudaStream_t s) {
  return gemm_path(0, ta, tb, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, s);
}

// ------------------------------------------------------------ elementwise
__device__ __forceinline__ float gelu_f(float x) {
  const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
  return 0.5f * x * (1.f + tanhf(u));
}
__device__ __forceinline__ float gelu_df(float x) {
  const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
  const float th = tanhf(u);
  return 0.5f * (1.f + th) + 0.5f * x * (1.f - th * th) * 0.7978845608028654f * (1.f + 3.f * 0.044715f * x * x);
}

#define GRID_STRIDE(q, n) for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (n); \
                               q += (long long)gridDim.x * blockDim.x)

__global__ void k_normalize(const float *X, const float *mean, const float *scale, int n, int d, __nv_bfloat16 *out) {
  GRID_STRIDE(q, (long long)n * d) out[q] = __float2bfloat16((X[q] - mean[q % d]) / scale[q % d]);
}

// pre = Z + bias (row-major [rows][N]), act = gelu(pre) as BF16
__global__ void k_bias_gelu(const float *Z, const float *bias, long long rows, int N, float *pre, __nv_bfloat16 *act) {
  GRID_STRIDE(q, rows * N) {
    const float v = Z[q] + bias[q % N];
    pre[q] = v;
    act[q] = __float2bfloat16(gelu_f(v));
  }
}

// y = Z + bias (final layer, FP32)
__global__ void k_bias(const float *Z, const float *bias, long long rows, int N, float *y) {
  GRID_STRIDE(q, rows * N) y[q] = Z[q] + bias[q % N];
}

// col2im of a transposed convolution (kernel 4, stride 2, padding 1):
// out[b][t][co] = bias[co] + sum over the taps (s, q) with 2 s - 1 + q = t of Z[b][s][co*4 + q]
__global__ void k_col2im(const float *Z, const float *bias, int B, int Lin, int Cout, float *pre,
                         __nv_bfloat16 *act) {
  const int Lout = 2 * Lin;
  GRID_STRIDE(q, (long long)B * Lout * Cout) {
    const int co = (int)(q % Cout);
    const long long bt = q / Cout;
    const int t = (int)(bt % Lout), b = (int)(bt / Lout);
    float v = bias[co];
    // t even: taps q = 1 (s = t/2), q = 3 (s = t/2 - 1); t odd: q = 0 (s = (t+1)/2), q = 2 (s = (t-1)/2)
    const int qa = (t & 1) ? 0 : 1, qb = qa + 2;
    const int sa = (t + 1 - qa) / 2, sb = (t + 1 - qb) / 2;
    if (sa >= 0 && sa < Lin) v += Z[((long long)b * Lin + sa) * (Cout * 4) + co * 4 + qa];
    if (sb >= 0 && sb < Lin) v += Z[((long long)b * Lin + sb) * (Cout * 4) + co * 4 + qb];
    pre[q] = v;
    act[q] = __float2bfloat16(gelu_f(v));
  }
}

// dz = da * gelu'(pre), FP32 and BF16 copies
__global__ void k_gelu_bwd(const float *da, const float *pre, long long n, float *dz, __nv_bfloat16 *dz16) {
  GRID_STRIDE(q, n) {
    const float v = da[q] * gelu_df(pre[q]);
    dz[q] = v;
    if (dz16) dz16[q] = __float2bfloat16(v);
  }
}

// im2col of the transposed convolution's gradient: dZ[b][s][co*4+q] = dy[b][2s-1+q][co]
__global__ void k_im2col(const float *dy, int B, int Lin, int Cout, __nv_bfloat16 *dZ) {
  const int Lout = 2 * Lin;
  GRID_STRIDE(q, (long long)B * Lin * Cout * 4) {
    const int cq = (int)(q % (Cout * 4));
    const long long bs = q / (Cout * 4);
    const int s = (int)(bs % Lin), b = (int)(bs / Lin);
    const int co = cq >> 2, tap = cq & 3, t = 2 * s - 1 + tap;
    dZ[q] = __float2bfloat16((t >= 0 && t < Lout) ? dy[((long long)b * Lout + t) * Cout + co] : 0.f);
  }
}

// column sums of a [rows][N] FP32 matrix into out[N] (fixed order: per-column
// partial sums over row blocks, then a sum of the partials)
__global__ void k_colsum_partial(const float *X, long long rows, int N, int chunk, float *part) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const long long r0 = (long long)blockIdx.y * chunk;
  if (n >= N) return;
  float acc = 0.f;
  for (long long r = r0; r < r0 + chunk && r < rows; r++) acc += X[r * N + n];
  part[(long long)blockIdx.y * N + n] = acc;
}
__global__ void k_colsum_final(const float *part, int parts, int N, float *out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int p = 0; p < parts; p++) acc += part[(long long)p * N + n];
  out[n] = acc;
}

// MSE of channels-last predictions y[b][t][c] against targets T[b][c][t]:
// loss partials per block, gradient dy = 2 (y - T) / count
__global__ void k_mse(const float *y, const float *T, int B, int L, int Cc, float inv_count, float inv_ys, float *dy,
                      float *loss_part) {
  __shared__ float red[256];
  float acc = 0.f;
  GRID_STRIDE(q, (long long)B * L * Cc) {
    const int c = (int)(q % Cc);
    const long long bt = q / Cc;
    const int t = (int)(bt % L), b = (int)(bt / L);
    const float e = y[q] - T[((long long)b * Cc + c) * L + t] * inv_ys;
    if (dy) dy[q] = 2.f * e * inv_count;
    acc += e * e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// channels-last [b][t][c] -> [b][c][t]
__global__ void k_to_channels_first(const float *y, int B, int L, int Cc, float scale, float *out) {
  GRID_STRIDE(q, (long long)B * L * Cc) {
    const int t = (int)(q % L);
    const long long bc = q / L;
    const int c = (int)(bc % Cc), b = (int)(bc / Cc);
    out[q] = y[((long long)b * L + t) * Cc + c] * scale;
  }
}

__global__ void k_to_bf16(const float *x, long long n, __nv_bfloat16 *y) {
  GRID_STRIDE(q, n) y[q] = __float2bfloat16(x[q]);
}

__global__ void k_adam(float *w, const float *g, float *m, float *v, __nv_bfloat16 *w16, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  GRID_STRIDE(q, n) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq, vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    w[q] = wq;
    w16[q] = __float2bfloat16(wq);
  }
}

// gather rows of the device training set into a minibatch
// per case b: num[b] = sum (y - y0)^2 and den[b] = sum y0^2 over its `per`
// outputs (one block per case, fixed-order tree in the block)
__global__ void __launch_bounds__(256) k_diff_norms(const float *y, const float *y0, long long per, float *num,
                                                    float *den) {
  const long long o = (long long)blockIdx.x * per;
  float a = 0.f, b = 0.f;
  for (long long q = threadIdx.x; q < per; q += 256) {
    const float u = y0[o + q], d = y[o + q] - u;
    a += d * d;
    b += u * u;
  }
  __shared__ float sa[256], sb[256];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    num[blockIdx.x] = sa[0];
    den[blockIdx.x] = sb[0];
  }
}

__global__ void k_gather(const float *src, const int *idx, int n, long long row, float *dst) {
  GRID_STRIDE(q, (long long)n * row) dst[q] = src[(long long)idx[q / row] * row + q % row];
}

static int egrid(long long n) { return (int)std::min<long long>((n + 255) / 256, 152 * 16); }

}  // namespace cwell

// ======================================================================= host
using namespace cwell;

struct sur_s {
  sur_cfg_t cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  long long nparam = 0;
  int max_batch = 0;
  std::vector<long long> off;  // parameter offsets: W1 b1 W2 b2 W3 b3 (T_l t_l)*nup Wf bf
  std::vector<int> chans;      // C0, C1, ..., C_nup
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *w16 = nullptr;
  float *x_mean = nullptr, *x_scale = nullptr;
  float y_scale = 1.f;  // outputs are y_scale times the network's (normalised) output
  long long adam_t = 0;
  // activations (sized for max_batch)
  std::vector<float *> pre;             // per layer pre-activations (FP32)
  std::vector<__nv_bfloat16 *> act;     // per layer activations (BF16), act[0] = normalised input
  float *z = nullptr, *y = nullptr, *dy = nullptr, *da = nullptr, *dz = nullptr, *part = nullptr, *lossp = nullptr;
  __nv_bfloat16 *dz16 = nullptr, *dy16 = nullptr;
  float *xb = nullptr, *tb = nullptr;
  int *idx = nullptr;
  std::vector<void *> allocs;
  std::vector<float> gate_x, gate_err;  // normalised validation inputs and their errors
  std::string err;
};

static thread_local std::string g_sur_err;
static int sfail(sur_t *s, int code, const std::string &m);

// a bounded wait of the tcgen05 GEMM that gave up surfaces as SIM_ETIMEOUT
static int tc_status(sur_t *s) {
  int st = 0;
  cudaError_t e = gemm_tcgen05_status(&st, s->stream);
  if (e != cudaSuccess) return sfail(s, SIM_ECUDA, cudaGetErrorString(e));
  if (st) return sfail(s, SIM_ETIMEOUT, "a tcgen05 GEMM wait gave up");
  return SIM_OK;
}

static int sfail(sur_t *s, int code, const std::string &m) {
  if (s) s->err = m;
  else g_sur_err = m;
  return code;
}

#define SCK(s, call)                                                                            \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return sfail(s, SIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename P>
static int salloc(sur_t *s, P **p, size_t bytes) {
  cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, SIM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  s->allocs.push_back(*p);
  return SIM_OK;
}

static int L_out(const sur_t *s) { return s->cfg.l0 << s->cfg.n_up; }

// layer widths: dense sizes and per-layer activation element counts
static void layout(sur_t *s) {
  const sur_cfg_t &c = s->cfg;
  s->chans.assign(c.chans, c.chans + c.n_up + 1);
  s->off.clear();
  long long o = 0;
  auto add = [&](long long n) {
    s->off.push_back(o);
    o += n;
  };
  add((long long)c.in_dim * c.h1);
  add(c.h1);
  add((long long)c.h1 * c.h2);
  add(c.h2);
  add((long long)c.h2 * c.l0 * c.chans[0]);
  add((long long)c.l0 * c.chans[0]);
  for (int l = 0; l < c.n_up; l++) {
    add((long long)c.chans[l] * c.chans[l + 1] * 4);
    add(c.chans[l + 1]);
  }
  add((long long)c.chans[c.n_up] * c.out_ch);
  add(c.out_ch);
  s->off.push_back(o);
  s->nparam = o;
}

extern "C" int sur_create(const sur_cfg_t *cfg, const sim_opts_t *opts, sur_t **out) {
  if (!out) return sfail(nullptr, SIM_EINVAL, "out is null");
  *out = nullptr;
  if (!cfg || cfg->in_dim < 1 || cfg->h1 < 1 || cfg->h2 < 1 || cfg->l0 < 1 || cfg->n_up < 0 || cfg->n_up > 8 ||
      cfg->out_ch < 1 || cfg->max_batch < 1)
    return sfail(nullptr, SIM_EINVAL, "bad surrogate configuration");
  for (int l = 0; l <= cfg->n_up; l++)
    if (cfg->chans[l] < 1) return sfail(nullptr, SIM_EINVAL, "bad channel count");
  sur_t *s = new sur_t();
  s->cfg = *cfg;
  s->max_batch = cfg->max_batch;
  s->device = opts ? opts->device : 0;
  auto bail = [&](int rc) {
    g_sur_err = s->err;
    for (void *p : s->allocs) cudaFree(p);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return rc;
  };
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return bail(sfail(s, SIM_ECUDA, cudaGetErrorString(e)));
  if (opts && opts->cuda_stream) {
    s->stream = (cudaStream_t)opts->cuda_stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(sfail(s, SIM_ECUDA, cudaGetErrorString(e)));
    s->own_stream = true;
  }
  layout(s);
  const long long P = s->nparam;
  int rc;
  if ((rc = salloc(s, &s->w, P * 4)) || (rc = salloc(s, &s->g, P * 4)) || (rc = salloc(s, &s->m, P * 4)) ||
      (rc = salloc(s, &s->v, P * 4)) || (rc = salloc(s, &s->w16, P * 2)) || (rc = salloc(s, &s->x_mean, cfg->in_dim * 4)) ||
      (rc = salloc(s, &s->x_scale, cfg->in_dim * 4)))
    return bail(rc);
  const int B = s->max_batch, Lf = L_out(s);
  // activations: layer 0 input, 1 h1, 2 h2, 3 a0 (= reshaped dense), 4.. convT outputs
  std::vector<long long> an = {(long long)B * cfg->in_dim, (long long)B * cfg->h1, (long long)B * cfg->h2,
                               (long long)B * cfg->l0 * cfg->chans[0]};
  long long zmax = std::max<long long>((long long)B * cfg->l0 * cfg->chans[0], (long long)B * Lf * cfg->out_ch);
  for (int l = 0; l < cfg->n_up; l++) {
    const long long Lin = (long long)cfg->l0 << l;
    an.push_back((long long)B * 2 * Lin * cfg->chans[l + 1]);
    zmax = std::max(zmax, (long long)B * Lin * cfg->chans[l + 1] * 4);
  }
  long long amax = 0;
  for (long long a : an) amax = std::max(amax, a);
  zmax = std::max(zmax, amax);
  s->pre.resize(an.size());
  s->act.resize(an.size());
  for (size_t l = 0; l < an.size(); l++) {
    if ((rc = salloc(s, &s->pre[l], an[l] * 4)) || (rc = salloc(s, &s->act[l], an[l] * 2))) return bail(rc);
  }
  if ((rc = salloc(s, &s->z, zmax * 4)) || (rc = salloc(s, &s->y, (long long)B * Lf * cfg->out_ch * 4)) ||
      (rc = salloc(s, &s->dy, (long long)B * Lf * cfg->out_ch * 4)) || (rc = salloc(s, &s->da, zmax * 4)) ||
      (rc = salloc(s, &s->dz, zmax * 4)) || (rc = salloc(s, &s->dz16, zmax * 2)) ||
      (rc = salloc(s, &s->dy16, zmax * 2)) || (rc = salloc(s, &s->part, 4096LL * 4096 * 4)) ||
      (rc = salloc(s, &s->lossp, 4096 * 4)) || (rc = salloc(s, &s->xb, (long long)B * cfg->in_dim * 4)) ||
      (rc = salloc(s, &s->tb, (long long)B * Lf * cfg->out_ch * 4)) || (rc = salloc(s, &s->idx, B * 4)))
    return bail(rc);
  // initial weights: uniform +-sqrt(6 / (fan_in + fan_out)) from SplitMix64, biases 0
  std::vector<float> w(P, 0.f);
  uint64_t st = cfg->seed;
  auto uni = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int slot, double fan_in, double fan_out) {
    const double a = sqrt(6.0 / (fan_in + fan_out));
    for (long long q = s->off[slot]; q < s->off[slot + 1]; q++) w[q] = (float)((2.0 * uni() - 1.0) * a);
  };
  fill(0, cfg->in_dim, cfg->h1);
  fill(2, cfg->h1, cfg->h2);
  fill(4, cfg->h2, (double)cfg->l0 * cfg->chans[0]);
  for (int l = 0; l < cfg->n_up; l++) fill(6 + 2 * l, 2.0 * cfg->chans[l], 2.0 * cfg->chans[l + 1]);
  fill(6 + 2 * cfg->n_up, cfg->chans[cfg->n_up], cfg->out_ch);
  std::vector<float> ones(cfg->in_dim, 1.f), zeros(cfg->in_dim, 0.f);
  if ((e = cudaMemcpy(s->w, w.data(), P * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(s->x_mean, zeros.data(), cfg->in_dim * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(s->x_scale, ones.data(), cfg->in_dim * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(s->m, 0, P * 4)) != cudaSuccess || (e = cudaMemset(s->v, 0, P * 4)) != cudaSuccess)
    return bail(sfail(s, SIM_ECUDA, cudaGetErrorString(e)));
  k_to_bf16<<<egrid(P), 256, 0, s->stream>>>(s->w, P, s->w16);
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return bail(sfail(s, SIM_ECUDA, cudaGetErrorString(e)));
  *out = s;
  return SIM_OK;
}

static float *Wp(sur_t *s, int slot) { return s->w + s->off[slot]; }
static __nv_bfloat16 *W16(sur_t *s, int slot) { return s->w16 + s->off[slot]; }
static float *Gp(sur_t *s, int slot) { return s->g + s->off[slot]; }

static cudaError_t colsum(sur_t *s, const float *X, long long rows, int N, float *out) {
  const int chunk = 256;
  const int parts = (int)std::min<long long>((rows + chunk - 1) / chunk, 4096);
  const int ch = (int)((rows + parts - 1) / parts);
  dim3 g1((N + 127) / 128, parts);
  k_colsum_partial<<<g1, 128, 0, s->stream>>>(X, rows, N, ch, s->part);
  k_colsum_final<<<(N + 127) / 128, 128, 0, s->stream>>>(s->part, parts, N, out);
  return cudaGetLastError();
}

// forward pass of n <= max_batch samples whose raw inputs are in s->xb
static cudaError_t forward(sur_t *s, int n) {
  const sur_cfg_t &c = s->cfg;
  cudaStream_t st = s->stream;
  cudaError_t e;
  k_normalize<<<egrid((long long)n * c.in_dim), 256, 0, st>>>(s->xb, s->x_mean, s->x_scale, n, c.in_dim, s->act[0]);
  const int dims[4] = {c.in_dim, c.h1, c.h2, c.l0 * c.chans[0]};
  for (int l = 0; l < 3; l++) {
    if ((e = gemm(false, false, n, dims[l + 1], dims[l], s->act[l], dims[l], W16(s, 2 * l), dims[l + 1], s->z,
                  dims[l + 1], 1.f, 0.f, st)) != cudaSuccess)
      return e;
    k_bias_gelu<<<egrid((long long)n * dims[l + 1]), 256, 0, st>>>(s->z, Wp(s, 2 * l + 1), n, dims[l + 1],
                                                                     s->pre[l + 1], s->act[l + 1]);
  }
  for (int l = 0; l < c.n_up; l++) {
    const int Lin = c.l0 << l, Cin = c.chans[l], Cout = c.chans[l + 1];
    const long long rows = (long long)n * Lin;
    if ((e = gemm(false, false, (int)rows, Cout * 4, Cin, s->act[3 + l], Cin, W16(s, 6 + 2 * l), Cout * 4, s->z,
                  Cout * 4, 1.f, 0.f, st)) != cudaSuccess)
      return e;
    k_col2im<<<egrid(rows * 2 * Cout), 256, 0, st>>>(s->z, Wp(s, 7 + 2 * l), n, Lin, Cout, s->pre[4 + l],
                                                      s->act[4 + l]);
  }
  const int Lf = L_out(s), Cl = c.chans[c.n_up];
  const long long rows = (long long)n * Lf;
  if ((e = gemm(false, false, (int)rows, c.out_ch, Cl, s->act[3 + c.n_up], Cl, W16(s, 6 + 2 * c.n_up), c.out_ch,
                s->z, c.out_ch, 1.f, 0.f, st)) != cudaSuccess)
    return e;
  k_bias<<<egrid(rows * c.out_ch), 256, 0, st>>>(s->z, Wp(s, 7 + 2 * c.n_up), rows, c.out_ch, s->y);
  return cudaGetLastError();
}

// loss (host value) and gradient into s->g for the targets in s->tb
static cudaError_t backward(sur_t *s, int n, float *loss_out) {
  const sur_cfg_t &c = s->cfg;
  cudaStream_t st = s->stream;
  cudaError_t e;
  const int Lf = L_out(s), Cl = c.chans[c.n_up];
  const long long rows = (long long)n * Lf, count = rows * c.out_ch;
  const int lblocks = 1024;
  k_mse<<<lblocks, 256, 0, st>>>(s->y, s->tb, n, Lf, c.out_ch, 1.f / (float)count, 1.f / s->y_scale, s->dy, s->lossp);
  if (loss_out) {
    std::vector<float> lp(lblocks);
    if ((e = cudaMemcpyAsync(lp.data(), s->lossp, lblocks * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    double acc = 0;
    for (float x : lp) acc += x;
    *loss_out = (float)(acc / (double)count);
  }
  // final 1x1 layer
  k_to_bf16<<<egrid(count), 256, 0, st>>>(s->dy, count, s->dy16);
  if ((e = gemm(true, false, Cl, c.out_ch, (int)rows, s->act[3 + c.n_up], Cl, s->dy16, c.out_ch,
                Gp(s, 6 + 2 * c.n_up), c.out_ch, 1.f, 0.f, st)) != cudaSuccess)
    return e;
  if ((e = colsum(s, s->dy, rows, c.out_ch, Gp(s, 7 + 2 * c.n_up))) != cudaSuccess) return e;
  if ((e = gemm(false, true, (int)rows, Cl, c.out_ch, s->dy16, c.out_ch, W16(s, 6 + 2 * c.n_up), c.out_ch, s->da, Cl,
                1.f, 0.f, st)) != cudaSuccess)
    return e;
  // transposed convolutions, last to first
  for (int l = c.n_up - 1; l >= 0; l--) {
    const int Lin = c.l0 << l, Cin = c.chans[l], Cout = c.chans[l + 1];
    const long long orow = (long long)n * 2 * Lin, irow = (long long)n * Lin;
    k_gelu_bwd<<<egrid(orow * Cout), 256, 0, st>>>(s->da, s->pre[4 + l], orow * Cout, s->dz, nullptr);
    if ((e = colsum(s, s->dz, orow, Cout, Gp(s, 7 + 2 * l))) != cudaSuccess) return e;
    k_im2col<<<egrid(irow * Cout * 4), 256, 0, st>>>(s->dz, n, Lin, Cout, s->dz16);
    if ((e = gemm(true, false, Cin, Cout * 4, (int)irow, s->act[3 + l], Cin, s->dz16, Cout * 4, Gp(s, 6 + 2 * l),
                  Cout * 4, 1.f, 0.f, st)) != cudaSuccess)
      return e;
    if ((e = gemm(false, true, (int)irow, Cin, Cout * 4, s->dz16, Cout * 4, W16(s, 6 + 2 * l), Cout * 4, s->da, Cin,
                  1.f, 0.f, st)) != cudaSuccess)
      return e;
  }
  // dense layers 3, 2, 1
  const int dims[4] = {c.in_dim, c.h1, c.h2, c.l0 * c.chans[0]};
  for (int l = 2; l >= 0; l--) {
    const long long nel = (long long)n * dims[l + 1];
    k_gelu_bwd<<<egrid(nel), 256, 0, st>>>(s->da, s->pre[l + 1], nel, s->dz, s->dz16);
    if ((e = colsum(s, s->dz, n, dims[l + 1], Gp(s, 2 * l + 1))) != cudaSuccess) return e;
    if ((e = gemm(true, false, dims[l], dims[l + 1], n, s->act[l], dims[l], s->dz16, dims[l + 1], Gp(s, 2 * l),
                  dims[l + 1], 1.f, 0.f, st)) != cudaSuccess)
      return e;
    if (l > 0 && (e = gemm(false, true, n, dims[l], dims[l + 1], s->dz16, dims[l + 1], W16(s, 2 * l), dims[l + 1],
                           s->da, dims[l], 1.f, 0.f, st)) != cudaSuccess)
      return e;
  }
  return cudaGetLastError();
}

extern "C" int sur_param_count(const sur_t *s, long long *n) {
  if (!s || !n) return SIM_EINVAL;
  *n = s->nparam;
  return SIM_OK;
}

extern "C" int sur_get_params(sur_t *s, float *out, size_t n) {
  if (!s || !out || n < (size_t)s->nparam) return s ? sfail(s, SIM_EINVAL, "buffer too small") : SIM_EINVAL;
  SCK(s, cudaStreamSynchronize(s->stream));
  SCK(s, cudaMemcpy(out, s->w, s->nparam * 4, cudaMemcpyDeviceToHost));
  return SIM_OK;
}

extern "C" int sur_set_params(sur_t *s, const float *in, size_t n) {
  if (!s || !in || n < (size_t)s->nparam) return s ? sfail(s, SIM_EINVAL, "buffer too small") : SIM_EINVAL;
  SCK(s, cudaStreamSynchronize(s->stream));
  SCK(s, cudaMemcpy(s->w, in, s->nparam * 4, cudaMemcpyHostToDevice));
  k_to_bf16<<<egrid(s->nparam), 256, 0, s->stream>>>(s->w, s->nparam, s->w16);
  SCK(s, cudaGetLastError());
  SCK(s, cudaMemset(s->m, 0, s->nparam * 4));
  SCK(s, cudaMemset(s->v, 0, s->nparam * 4));
  s->adam_t = 0;
  return SIM_OK;
}

extern "C" int sur_set_normalization(sur_t *s, const float *x_mean, const float *x_scale, float y_scale) {
  if (!s || !x_mean || !x_scale) return SIM_EINVAL;
  if (!(y_scale > 0) || !isfinite(y_scale)) return sfail(s, SIM_EINVAL, "output scale must be positive and finite");
  s->y_scale = y_scale;
  SCK(s, cudaStreamSynchronize(s->stream));
  for (int q = 0; q < s->cfg.in_dim; q++)
    if (!(x_scale[q] != 0.f) || !isfinite(x_scale[q]) || !isfinite(x_mean[q]))
      return sfail(s, SIM_EINVAL, "normalisation scales must be finite and non-zero");
  SCK(s, cudaMemcpy(s->x_mean, x_mean, s->cfg.in_dim * 4, cudaMemcpyHostToDevice));
  SCK(s, cudaMemcpy(s->x_scale, x_scale, s->cfg.in_dim * 4, cudaMemcpyHostToDevice));
  return SIM_OK;
}

extern "C" int sur_forward(sur_t *s, const float *X, int n, float *Y) {
  if (!s || n < 0 || (n > 0 && (!X || !Y))) return s ? sfail(s, SIM_EINVAL, "bad arguments") : SIM_EINVAL;
  SCK(s, cudaSetDevice(s->device));
  const sur_cfg_t &c = s->cfg;
  const int Lf = L_out(s);
  std::vector<float> tmp((size_t)s->max_batch * Lf * c.out_ch);
  for (int b0 = 0; b0 < n; b0 += s->max_batch) {
    const int nb = std::min(s->max_batch, n - b0);
    SCK(s, cudaMemcpyAsync(s->xb, X + (size_t)b0 * c.in_dim, (size_t)nb * c.in_dim * 4, cudaMemcpyHostToDevice,
                           s->stream));
    SCK(s, forward(s, nb));
    k_to_channels_first<<<egrid((long long)nb * Lf * c.out_ch), 256, 0, s->stream>>>(s->y, nb, Lf, c.out_ch,
                                                                                     s->y_scale, s->dz);
    SCK(s, cudaGetLastError());
    SCK(s, cudaMemcpyAsync(Y + (size_t)b0 * Lf * c.out_ch, s->dz, (size_t)nb * Lf * c.out_ch * 4,
                           cudaMemcpyDeviceToHost, s->stream));
  }
  SCK(s, cudaStreamSynchronize(s->stream));
  return tc_status(s);
}

extern "C" int sur_sensitivity(sur_t *s, const float *X, int n, float step, float *sens) {
  if (!s || n < 0 || (n > 0 && (!X || !sens)) || !(step > 0.f))
    return s ? sfail(s, SIM_EINVAL, "bad arguments") : SIM_EINVAL;
  SCK(s, cudaSetDevice(s->device));
  const sur_cfg_t &c = s->cfg;
  const long long per = (long long)L_out(s) * c.out_ch;
  std::vector<float> scale(c.in_dim), xp((size_t)s->max_batch * c.in_dim), num(s->max_batch), den(s->max_batch);
  SCK(s, cudaMemcpy(scale.data(), s->x_scale, c.in_dim * 4, cudaMemcpyDeviceToHost));
  float *nd = s->part;  // [2][max_batch] partial norms (the column-sum scratch, idle here)
  for (int b0 = 0; b0 < n; b0 += s->max_batch) {
    const int nb = std::min(s->max_batch, n - b0);
    const float *xc = X + (size_t)b0 * c.in_dim;
    SCK(s, cudaMemcpyAsync(s->xb, xc, (size_t)nb * c.in_dim * 4, cudaMemcpyHostToDevice, s->stream));
    SCK(s, forward(s, nb));
    SCK(s, cudaMemcpyAsync(s->dy, s->y, (size_t)nb * per * 4, cudaMemcpyDeviceToDevice, s->stream));
    for (int q = 0; q < nb; q++) sens[b0 + q] = 0.f;
    for (int d = 0; d < c.in_dim; d++) {
      // the input moved by `step` in normalised units along dimension d
      for (int q = 0; q < nb; q++)
        for (int e = 0; e < c.in_dim; e++)
          xp[(size_t)q * c.in_dim + e] = xc[(size_t)q * c.in_dim + e] + (e == d ? step * scale[d] : 0.f);
      SCK(s, cudaMemcpyAsync(s->xb, xp.data(), (size_t)nb * c.in_dim * 4, cudaMemcpyHostToDevice, s->stream));
      SCK(s, forward(s, nb));
      k_diff_norms<<<nb, 256, 0, s->stream>>>(s->y, s->dy, per, nd, nd + s->max_batch);
      SCK(s, cudaGetLastError());
      SCK(s, cudaMemcpyAsync(num.data(), nd, nb * 4, cudaMemcpyDeviceToHost, s->stream));
      SCK(s, cudaMemcpyAsync(den.data(), nd + s->max_batch, nb * 4, cudaMemcpyDeviceToHost, s->stream));
      SCK(s, cudaStreamSynchronize(s->stream));
      for (int q = 0; q < nb; q++)
        sens[b0 + q] = std::max(sens[b0 + q], den[q] > 0.f ? std::sqrt(num[q] / den[q]) : INFINITY);
    }
  }
  return tc_status(s);
}

extern "C" int sur_loss_grad(sur_t *s, const float *X, const float *Y, int n, float *loss, float *grad, size_t ng) {
  if (!s || !X || !Y || n < 1 || n > s->max_batch) return s ? sfail(s, SIM_EINVAL, "bad arguments") : SIM_EINVAL;
  if (grad && ng < (size_t)s->nparam) return sfail(s, SIM_EINVAL, "gradient buffer too small");
  const sur_cfg_t &c = s->cfg;
  const int Lf = L_out(s);
  SCK(s, cudaMemcpyAsync(s->xb, X, (size_t)n * c.in_dim * 4, cudaMemcpyHostToDevice, s->stream));
  SCK(s, cudaMemcpyAsync(s->tb, Y, (size_t)n * Lf * c.out_ch * 4, cudaMemcpyHostToDevice, s->stream));
  SCK(s, forward(s, n));
  float l = 0.f;
  SCK(s, backward(s, n, &l));
  if (loss) *loss = l;
  // the gradient kernels run on the handle's (non-blocking) stream: copy on it and wait
  if (grad) SCK(s, cudaMemcpyAsync(grad, s->g, s->nparam * 4, cudaMemcpyDeviceToHost, s->stream));
  SCK(s, cudaStreamSynchronize(s->stream));
  return tc_status(s);
}

extern "C" int sur_train(sur_t *s, const float *X, const float *Y, int n, int epochs, int batch, float lr,
                         unsigned long long seed, float *epoch_loss) {
  if (!s || !X || !Y || n < 1 || epochs < 0 || batch < 1 || batch > s->max_batch || !(lr > 0))
    return s ? sfail(s, SIM_EINVAL, "bad training arguments") : SIM_EINVAL;
  SCK(s, cudaSetDevice(s->device));
  const sur_cfg_t &c = s->cfg;
  const int Lf = L_out(s);
  const long long xrow = c.in_dim, yrow = (long long)Lf * c.out_ch;
  float *dX = nullptr, *dY = nullptr;
  SCK(s, cudaMalloc(&dX, (size_t)n * xrow * 4));
  cudaError_t e = cudaMalloc(&dY, (size_t)n * yrow * 4);
  if (e != cudaSuccess) {
    cudaFree(dX);
    return sfail(s, SIM_ENOMEM, cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(dX, X, (size_t)n * xrow * 4, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dY, Y, (size_t)n * yrow * 4, cudaMemcpyHostToDevice, s->stream);
  std::vector<int> perm(n);
  for (int q = 0; q < n; q++) perm[q] = q;
  uint64_t st = seed;
  auto rnd = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  const long long steps_total = (long long)epochs * ((n + batch - 1) / batch);
  long long step = 0;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ep++) {
    for (int q = n - 1; q > 0; q--) std::swap(perm[q], perm[rnd() % (uint64_t)(q + 1)]);
    double lsum = 0;
    int nb_count = 0;
    for (int b0 = 0; b0 < n && e == cudaSuccess; b0 += batch) {
      const int nb = std::min(batch, n - b0);
      e = cudaMemcpyAsync(s->idx, perm.data() + b0, nb * 4, cudaMemcpyHostToDevice, s->stream);
      if (e != cudaSuccess) break;
      k_gather<<<egrid(nb * xrow), 256, 0, s->stream>>>(dX, s->idx, nb, xrow, s->xb);
      k_gather<<<egrid(nb * yrow), 256, 0, s->stream>>>(dY, s->idx, nb, yrow, s->tb);
      if ((e = forward(s, nb)) != cudaSuccess) break;
      float l = 0.f;
      if ((e = backward(s, nb, &l)) != cudaSuccess) break;
      lsum += l;
      nb_count++;
      // cosine learning-rate schedule over all steps
      const float lr_t = 0.5f * lr * (1.f + cosf(3.14159265f * (float)step / (float)std::max<long long>(1, steps_total)));
      s->adam_t++;
      step++;
      const float c1 = 1.f - powf(b1, (float)s->adam_t), c2 = 1.f - powf(b2, (float)s->adam_t);
      k_adam<<<egrid(s->nparam), 256, 0, s->stream>>>(s->w, s->g, s->m, s->v, s->w16, s->nparam, lr_t, b1, b2, eps, c1,
                                                       c2);
      e = cudaGetLastError();
    }
    if (epoch_loss) epoch_loss[ep] = (float)(lsum / std::max(1, nb_count));
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(dX);
  cudaFree(dY);
  if (e != cudaSuccess) return sfail(s, SIM_ECUDA, cudaGetErrorString(e));
  return tc_status(s);
}

// fallback gate: errors of validation cases indexed by their normalised inputs
extern "C" int sur_gate_fit(sur_t *s, const float *X, const float *err, int n) {
  if (!s || n < 1 || !X || !err) return s ? sfail(s, SIM_EINVAL, "bad gate data") : SIM_EINVAL;
  const int d = s->cfg.in_dim;
  std::vector<float> mean(d), scale(d);
  SCK(s, cudaStreamSynchronize(s->stream));
  SCK(s, cudaMemcpy(mean.data(), s->x_mean, d * 4, cudaMemcpyDeviceToHost));
  SCK(s, cudaMemcpy(scale.data(), s->x_scale, d * 4, cudaMemcpyDeviceToHost));
  s->gate_x.resize((size_t)n * d);
  s->gate_err.assign(err, err + n);
  for (int q = 0; q < n; q++)
    for (int c = 0; c < d; c++) s->gate_x[(size_t)q * d + c] = (X[(size_t)q * d + c] - mean[c]) / scale[c];
  return SIM_OK;
}

// accept[q] = 1 when the largest error among the k validation cases nearest
// to input q (normalised Euclidean distance) is <= tol
extern "C" int sur_gate(sur_t *s, const float *X, int n, int k, float tol, int *accept) {
  if (!s || n < 0 || (n > 0 && (!X || !accept)) || k < 1) return s ? sfail(s, SIM_EINVAL, "bad gate query") : SIM_EINVAL;
  if (s->gate_err.empty()) return sfail(s, SIM_EINVAL, "gate not fitted");
  const int d = s->cfg.in_dim, m = (int)s->gate_err.size();
  std::vector<float> mean(d), scale(d);
  SCK(s, cudaMemcpy(mean.data(), s->x_mean, d * 4, cudaMemcpyDeviceToHost));
  SCK(s, cudaMemcpy(scale.data(), s->x_scale, d * 4, cudaMemcpyDeviceToHost));
  std::vector<std::pair<float, float>> dist(m);
  for (int q = 0; q < n; q++) {
    for (int j = 0; j < m; j++) {
      float acc = 0;
      for (int c = 0; c < d; c++) {
        const float u = (X[(size_t)q * d + c] - mean[c]) / scale[c] - s->gate_x[(size_t)j * d + c];
        acc += u * u;
      }
      dist[j] = {acc, s->gate_err[j]};
    }
    const int kk = std::min(k, m);
    std::partial_sort(dist.begin(), dist.begin() + kk, dist.end());
    float worst = 0;
    for (int j = 0; j < kk; j++) worst = std::max(worst, dist[j].second);
    accept[q] = worst <= tol ? 1 : 0;
  }
  return SIM_OK;
}

extern "C" void sur_destroy(sur_t *s) {
  if (!s) return;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (void *p : s->allocs) cudaFree(p);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

extern "C" const char *sur_last_error(const sur_t *s) { return s ? s->err.c_str() : g_sur_err.c_str(); }

// tensor-core GEMM on host buffers (BF16 bit patterns in, FP32 out)
extern "C" int cw_gemm_bf16(int trans_a, int trans_b, int M, int N, int K, const uint16_t *A, int lda,
                            const uint16_t *B, int ldb, float *C, int ldc) {
  return cw_gemm_bf16_path(0, trans_a, trans_b, M, N, K, A, lda, B, ldb, C, ldc);
}

extern "C" int cw_gemm_bf16_path(int path, int trans_a, int trans_b, int M, int N, int K, const uint16_t *A, int lda,
                                 const uint16_t *B, int ldb, float *C, int ldc) {
  if (path < 0 || path > 2 || M < 0 || N < 0 || K < 0 || !A || !B || !C) return SIM_EINVAL;
  const size_t na = (size_t)(trans_a ? K : M) * lda, nb = (size_t)(trans_b ? N : K) * ldb, nc = (size_t)M * ldc;
  __nv_bfloat16 *dA = nullptr, *dB = nullptr;
  float *dC = nullptr;
  cudaError_t e = cudaMalloc(&dA, std::max<size_t>(na, 1) * 2);
  if (e == cudaSuccess) e = cudaMalloc(&dB, std::max<size_t>(nb, 1) * 2);
  if (e == cudaSuccess) e = cudaMalloc(&dC, std::max<size_t>(nc, 1) * 4);
  if (e == cudaSuccess) e = cudaMemcpy(dA, A, na * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dB, B, nb * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = gemm_path(path, trans_a != 0, trans_b != 0, M, N, K, dA, lda, dB, ldb, dC, ldc, 1.f, 0.f, 0);
  if (e == cudaSuccess) e = cudaMemcpy(C, dC, nc * 4, cudaMemcpyDeviceToHost);
  int st = 0;
  if (e == cudaSuccess) e = gemm_tcgen05_status(&st, 0);
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  if (e != cudaSuccess) return SIM_ECUDA;
  return st ? SIM_ETIMEOUT : SIM_OK;
}
