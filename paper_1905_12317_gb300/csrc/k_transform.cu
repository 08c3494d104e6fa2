// Pixel images -> Fourier--Bessel coefficients (FP32 SIMT).
//
// eq. (Ahattrap): Ahat(k) = dx^2 sum_{i,j} A_ij exp(-i k . x_ij) on the polar grid
// (k_m, psi_p), psi_p = pi p / Q (Section 3.2). The sum is separable:
//   T_i(P) = sum_j A_ij Ey[j][P],  Ahat(P) = dx^2 sum_i Ex[i][P] T_i(P),
// with Ex/Ey the per-axis phase tables computed in FP64 on the host. Real
// images satisfy Ahat(k, psi + pi) = conj Ahat(k, psi), so only p < Q is summed
// and the other half is its conjugate.
// eq. (aqkcalc): the ring DFT a(k_m; q) = (1/2Q) sum_p Ahat(k_m, psi_p) e^{-i q psi_p}
// is then a batched length-2Q FFT over the rows of [B][M][2Q].
#include "fft.cuh"
#include "ftk_internal.h"

namespace ftk {

namespace {

template <int IB>
__global__ void __launch_bounds__(128) k_polar(const float* __restrict__ images, int B, int n,
                                               const float2* __restrict__ Ex, const float2* __restrict__ Ey,
                                               int MQ, int Q, float dx2, float2* __restrict__ out) {
  extern __shared__ float smem[];
  const int TP = blockDim.x;
  float* img = smem;                                    // [IB][n][n]
  float2* eys = reinterpret_cast<float2*>(img + IB * n * n);  // [n][TP]
  const int b0 = blockIdx.y * IB;
  const int P0 = blockIdx.x * TP;
  const int P = P0 + threadIdx.x;
  const int nimg = min(IB, B - b0);
  for (int e = threadIdx.x; e < IB * n * n; e += TP) {
    const int b = e / (n * n);
    img[e] = b < nimg ? images[static_cast<size_t>(b0 + b) * n * n + (e - b * n * n)] : 0.f;
  }
  for (int e = threadIdx.x; e < n * TP; e += TP) {
    const int j = e / TP, t = e - j * TP;
    eys[e] = (P0 + t < MQ) ? Ey[static_cast<size_t>(j) * MQ + P0 + t] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (P >= MQ) return;
  float2 acc[IB];
#pragma unroll
  for (int b = 0; b < IB; ++b) acc[b] = make_float2(0.f, 0.f);
  for (int i = 0; i < n; ++i) {
    float2 T[IB];
#pragma unroll
    for (int b = 0; b < IB; ++b) T[b] = make_float2(0.f, 0.f);
    const float* row = img + i * n;
    for (int j = 0; j < n; ++j) {
      const float2 e = eys[j * TP + threadIdx.x];
#pragma unroll
      for (int b = 0; b < IB; ++b) {
        const float v = row[b * n * n + j];
        T[b].x = fmaf(v, e.x, T[b].x);
        T[b].y = fmaf(v, e.y, T[b].y);
      }
    }
    const float2 ex = Ex[static_cast<size_t>(i) * MQ + P];
#pragma unroll
    for (int b = 0; b < IB; ++b) acc[b] = cadd(acc[b], cmul(ex, T[b]));
  }
  const int m = P / Q, p = P - m * Q;
  const int two_Q = 2 * Q;
#pragma unroll
  for (int b = 0; b < IB; ++b) {
    if (b < nimg) {
      float2* o = out + (static_cast<size_t>(b0 + b) * (MQ / Q) + m) * two_Q;
      const float2 v = make_float2(dx2 * acc[b].x, dx2 * acc[b].y);
      o[p] = v;
      o[p + Q] = make_float2(v.x, -v.y);
    }
  }
}

__global__ void k_fft_rows(float2* __restrict__ rows, long long nrows, int L, int rows_per_block,
                           FftSchedule sch, const float2* __restrict__ tw_g, float scale) {
  extern __shared__ float2 sh[];
  float2* tw = sh;                       // [L]
  float2* b0 = sh + L;                   // [rows_per_block * L]
  float2* b1 = b0 + rows_per_block * L;
  const long long r0 = static_cast<long long>(blockIdx.x) * rows_per_block;
  const int T = static_cast<int>(min(static_cast<long long>(rows_per_block), nrows - r0));
  for (int e = threadIdx.x; e < L; e += blockDim.x) tw[e] = tw_g[e];
  const float2* src = rows + r0 * L;
  for (int e = threadIdx.x; e < T * L; e += blockDim.x) b0[e] = src[e];
  __syncthreads();
  float2* res = stockham_fft(b0, b1, T, L, sch.radix, sch.n, tw);
  float2* dst = rows + r0 * L;
  for (int e = threadIdx.x; e < T * L; e += blockDim.x) {
    const float2 v = res[e];
    dst[e] = make_float2(v.x * scale, v.y * scale);
  }
}

// Rows of length L = 32 c: one warp per row, register FFT (warp_fft), result
// staged through shared memory so that loads and stores are coalesced.
template <int L>
__global__ void __launch_bounds__(256) k_fft_rows_w(float2* __restrict__ rows, long long nrows,
                                                    const float2* __restrict__ tw_g, float scale) {
  constexpr int c = L / 32;
  extern __shared__ float2 sh[];
  float2* tw = sh;
  float2* stage = sh + L + (threadIdx.x >> 5) * L;
  for (int e = threadIdx.x; e < L; e += blockDim.x) tw[e] = tw_g[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long row = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= nrows) return;
  float2* r = rows + row * L;
  float2 v[c];
#pragma unroll
  for (int k = 0; k < c; ++k) v[k] = r[lane + 32 * k];
  warp_fft<L>(v, tw);
  const int br = __brev(lane) >> 27;
#pragma unroll
  for (int f2 = 0; f2 < c; ++f2) stage[f2 + c * br] = make_float2(v[f2].x * scale, v[f2].y * scale);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < c; ++k) r[lane + 32 * k] = stage[lane + 32 * k];
}

template <int L>
cudaError_t launch_fft_rows_w(const ftk_plan_s* p, float2* d_rows, long long nrows, float scale, cudaStream_t s) {
  const size_t smem = static_cast<size_t>(L) * 9 * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_fft_rows_w<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long blocks = (nrows + 7) / 8;
  k_fft_rows_w<L><<<static_cast<unsigned>(blocks), 256, smem, s>>>(d_rows, nrows, p->d_tw, scale);
  return cudaGetLastError();
}

}  // namespace

FftSchedule make_fft_schedule(int L) {
  FftSchedule s;
  s.L = L;
  int r = L;
  while (r % 4 == 0) { s.radix[s.n++] = 4; r /= 4; }
  while (r % 2 == 0) { s.radix[s.n++] = 2; r /= 2; }
  while (r % 3 == 0) { s.radix[s.n++] = 3; r /= 3; }
  if (r != 1) s.n = -1;
  return s;
}

cudaError_t launch_polar_transform(const ftk_plan_s* p, const float* d_images, int B, float2* d_out,
                                   cudaStream_t s) {
  const int n = p->n, MQ = p->M * p->Q;
  int IB, TP;
  if (n <= 32) { IB = 8; TP = 128; }
  else if (n <= 64) { IB = 4; TP = 128; }
  else if (n <= 128) { IB = 1; TP = 128; }
  else { IB = 1; TP = 32; }
  const size_t smem = static_cast<size_t>(IB) * n * n * sizeof(float) + static_cast<size_t>(n) * TP * sizeof(float2);
  dim3 grid((MQ + TP - 1) / TP, (B + IB - 1) / IB);
  const float dx2 = static_cast<float>(p->dx * p->dx);
  cudaError_t e;
#define FTK_POLAR(IBV)                                                                                   \
  e = cudaFuncSetAttribute(k_polar<IBV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
  if (e != cudaSuccess) return e;                                                                        \
  k_polar<IBV><<<grid, TP, smem, s>>>(d_images, B, n, p->d_Ex, p->d_Ey, MQ, p->Q, dx2, d_out);
  if (IB == 8) { FTK_POLAR(8) } else if (IB == 4) { FTK_POLAR(4) } else { FTK_POLAR(1) }
#undef FTK_POLAR
  return cudaGetLastError();
}

cudaError_t launch_fft_rows(const ftk_plan_s* p, float2* d_rows, long long nrows, float scale,
                            cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  switch (p->two_Q) {
    case 96: return launch_fft_rows_w<96>(p, d_rows, nrows, scale, s);
    case 192: return launch_fft_rows_w<192>(p, d_rows, nrows, scale, s);
    case 288: return launch_fft_rows_w<288>(p, d_rows, nrows, scale, s);
    case 384: return launch_fft_rows_w<384>(p, d_rows, nrows, scale, s);
    case 576: return launch_fft_rows_w<576>(p, d_rows, nrows, scale, s);
    default: break;
  }
  const int L = p->two_Q;
  int rpb = (4096 + L - 1) / L;
  if (rpb < 1) rpb = 1;
  const size_t smem = static_cast<size_t>(L) * (2 * rpb + 1) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long blocks = (nrows + rpb - 1) / rpb;
  k_fft_rows<<<static_cast<unsigned>(blocks), 256, smem, s>>>(d_rows, nrows, L, rpb, p->fft, p->d_tw, scale);
  return cudaGetLastError();
}

}  // namespace ftk
