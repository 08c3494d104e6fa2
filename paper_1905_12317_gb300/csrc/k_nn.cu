// Template-proposal network: forward and backward kernels (FP32), its loss,
// Adam, top-k selection and a row gather. The paper has no counterpart; the
// network shortlists templates and a shift window for the FTK search.
// Layouts: activations NCHW contiguous, weights [Co][Ci][3][3], linear weights [O][I].
#include <cuda_runtime.h>

#include <cfloat>

#include "fft.cuh"
#include "ftk_internal.h"

namespace {

__global__ void k_nn_features(const float2* __restrict__ a, int B, int M, int two_Q, float eps_f,
                              float* __restrict__ x0, float* __restrict__ lin) {
  const int Q = two_Q / 2;
  const long long total = static_cast<long long>(B) * M * Q;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(e % Q);
    const long long bm = e / Q;  // b * M + m
    const float2 c = a[bm * two_Q + q];
    x0[e] = logf(eps_f + sqrtf(c.x * c.x + c.y * c.y));
    if (q < 2) {
      const int b = static_cast<int>(bm / M), m = static_cast<int>(bm % M);
      lin[static_cast<size_t>(b) * 4 * M + (2 * q) * M + m] = c.x;
      lin[static_cast<size_t>(b) * 4 * M + (2 * q + 1) * M + m] = c.y;
    }
  }
}

__global__ void k_conv3x3(const float* __restrict__ x, const float* __restrict__ w, const float* __restrict__ bias,
                          float* __restrict__ y, int B, int Ci, int Co, int H, int W, int relu) {
  const long long total = static_cast<long long>(B) * Co * H * W;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int ww = static_cast<int>(e % W);
    long long r = e / W;
    const int hh = static_cast<int>(r % H);
    r /= H;
    const int co = static_cast<int>(r % Co);
    const int b = static_cast<int>(r / Co);
    float acc = bias[co];
    const float* xb = x + static_cast<size_t>(b) * Ci * H * W;
    const float* wc = w + static_cast<size_t>(co) * Ci * 9;
    for (int ci = 0; ci < Ci; ++ci) {
      const float* xc = xb + static_cast<size_t>(ci) * H * W;
      const float* wk = wc + ci * 9;
#pragma unroll
      for (int kh = 0; kh < 3; ++kh) {
        const int h = hh + kh - 1;
        if (h < 0 || h >= H) continue;
#pragma unroll
        for (int kw = 0; kw < 3; ++kw) {
          const int v = ww + kw - 1;
          if (v < 0 || v >= W) continue;
          acc = fmaf(__ldg(wk + kh * 3 + kw), xc[h * W + v], acc);
        }
      }
    }
    y[e] = relu ? fmaxf(acc, 0.f) : acc;
  }
}

// dx[b][ci][h][w] = sum_{co,kh,kw} w[co][ci][kh][kw] dz[b][co][h+1-kh][w+1-kw]
__global__ void k_conv3x3_bwd_data(const float* __restrict__ w, const float* __restrict__ dz, float* __restrict__ dx,
                                   int B, int Ci, int Co, int H, int W) {
  const long long total = static_cast<long long>(B) * Ci * H * W;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int ww = static_cast<int>(e % W);
    long long r = e / W;
    const int hh = static_cast<int>(r % H);
    r /= H;
    const int ci = static_cast<int>(r % Ci);
    const int b = static_cast<int>(r / Ci);
    float acc = 0.f;
    for (int co = 0; co < Co; ++co) {
      const float* dzc = dz + (static_cast<size_t>(b) * Co + co) * H * W;
      const float* wk = w + (static_cast<size_t>(co) * Ci + ci) * 9;
#pragma unroll
      for (int kh = 0; kh < 3; ++kh) {
        const int h = hh + 1 - kh;
        if (h < 0 || h >= H) continue;
#pragma unroll
        for (int kw = 0; kw < 3; ++kw) {
          const int v = ww + 1 - kw;
          if (v < 0 || v >= W) continue;
          acc = fmaf(__ldg(wk + kh * 3 + kw), dzc[h * W + v], acc);
        }
      }
    }
    dx[e] = acc;
  }
}

// One block per (co, ci): dw[co][ci][kh][kw] = sum_{b,h,w} dz[b][co][h][w] x[b][ci][h+kh-1][w+kw-1];
// blocks with ci == 0 also produce db[co].
__global__ void __launch_bounds__(256) k_conv3x3_bwd_weight(const float* __restrict__ x, const float* __restrict__ dz,
                                                            float* __restrict__ dw, float* __restrict__ db, int B,
                                                            int Ci, int Co, int H, int W) {
  const int co = blockIdx.x / Ci, ci = blockIdx.x % Ci;
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
  const long long total = static_cast<long long>(B) * H * W;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int ww = static_cast<int>(e % W);
    const long long r = e / W;
    const int hh = static_cast<int>(r % H);
    const int b = static_cast<int>(r / H);
    const float g = dz[((static_cast<size_t>(b) * Co + co) * H + hh) * W + ww];
    const float* xc = x + (static_cast<size_t>(b) * Ci + ci) * H * W;
#pragma unroll
    for (int kh = 0; kh < 3; ++kh) {
      const int h = hh + kh - 1;
#pragma unroll
      for (int kw = 0; kw < 3; ++kw) {
        const int v = ww + kw - 1;
        if (h >= 0 && h < H && v >= 0 && v < W) acc[kh * 3 + kw] = fmaf(g, xc[h * W + v], acc[kh * 3 + kw]);
      }
    }
    acc[9] += g;
  }
  __shared__ float red[10][256];
#pragma unroll
  for (int k = 0; k < 10; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < 10; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 9) dw[(static_cast<size_t>(co) * Ci + ci) * 9 + threadIdx.x] = red[threadIdx.x][0];
  if (threadIdx.x == 9 && ci == 0 && db) db[co] = red[9][0];
}

// dy <- dy * (y > 0), y being the post-ReLU output
__global__ void k_relu_bwd(const float* __restrict__ y, float* __restrict__ dy, long long n) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x)
    if (!(y[e] > 0.f)) dy[e] = 0.f;
}

__global__ void k_pool2(const float* __restrict__ x, float* __restrict__ y, long long BC, int H, int W) {
  const int Ho = H / 2, Wo = W / 2;
  const long long total = BC * Ho * Wo;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int wo = static_cast<int>(e % Wo);
    const long long r = e / Wo;
    const int ho = static_cast<int>(r % Ho);
    const long long bc = r / Ho;
    const float* p = x + (bc * H + 2 * ho) * W + 2 * wo;
    y[e] = 0.25f * (p[0] + p[1] + p[W] + p[W + 1]);
  }
}

__global__ void k_pool2_bwd(const float* __restrict__ dy, float* __restrict__ dx, long long BC, int H, int W) {
  const long long total = BC * H * W;
  const int Wo = W / 2, Ho = H / 2;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int w = static_cast<int>(e % W);
    const long long r = e / W;
    const int h = static_cast<int>(r % H);
    const long long bc = r / H;
    dx[e] = 0.25f * dy[(bc * Ho + h / 2) * Wo + w / 2];
  }
}

__global__ void k_gap(const float* __restrict__ x, float* __restrict__ y, long long BC, int HW) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < BC;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < HW; ++k) s += x[e * HW + k];
    y[e] = s / HW;
  }
}

__global__ void k_gap_bwd(const float* __restrict__ dy, float* __restrict__ dx, long long BC, int HW) {
  const long long total = BC * HW;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x)
    dx[e] = dy[e / HW] / HW;
}

// y[b][o] = sum_i x[b][i] w[o][i] + bias[o] (optionally ReLU); x rows may be a
// concatenation of two inputs (x1 [B][I1] then x2 [B][I - I1]).
__global__ void k_linear(const float* __restrict__ x1, const float* __restrict__ x2, int I1,
                         const float* __restrict__ w, const float* __restrict__ bias, float* __restrict__ y, int B,
                         int I, int O, int relu) {
  const long long total = static_cast<long long>(B) * O;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int o = static_cast<int>(e % O);
    const int b = static_cast<int>(e / O);
    const float* wr = w + static_cast<size_t>(o) * I;
    float acc = bias[o];
    const float* xa = x1 + static_cast<size_t>(b) * I1;
    for (int i = 0; i < I1; ++i) acc = fmaf(xa[i], __ldg(wr + i), acc);
    if (x2) {
      const float* xb = x2 + static_cast<size_t>(b) * (I - I1);
      for (int i = I1; i < I; ++i) acc = fmaf(xb[i - I1], __ldg(wr + i), acc);
    }
    y[e] = relu ? fmaxf(acc, 0.f) : acc;
  }
}

// dx[b][i] = sum_o dy[b][o] w[o][i] (first I1 columns only when dx covers only x1)
__global__ void k_linear_bwd_data(const float* __restrict__ dy, const float* __restrict__ w, float* __restrict__ dx,
                                  int B, int I, int O, int Iout) {
  const long long total = static_cast<long long>(B) * Iout;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e % Iout);
    const int b = static_cast<int>(e / Iout);
    float acc = 0.f;
    for (int o = 0; o < O; ++o) acc = fmaf(dy[static_cast<size_t>(b) * O + o], __ldg(w + static_cast<size_t>(o) * I + i), acc);
    dx[e] = acc;
  }
}

// dw[o][i] = sum_b dy[b][o] x[b][i];  db[o] = sum_b dy[b][o]
__global__ void k_linear_bwd_weight(const float* __restrict__ x1, const float* __restrict__ x2, int I1,
                                    const float* __restrict__ dy, float* __restrict__ dw, float* __restrict__ db,
                                    int B, int I, int O) {
  const long long total = static_cast<long long>(O) * (I + 1);
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e % (I + 1));
    const int o = static_cast<int>(e / (I + 1));
    float acc = 0.f;
    if (i == I) {
      for (int b = 0; b < B; ++b) acc += dy[static_cast<size_t>(b) * O + o];
      db[o] = acc;
    } else {
      for (int b = 0; b < B; ++b) {
        const float xv = i < I1 ? x1[static_cast<size_t>(b) * I1 + i] : x2[static_cast<size_t>(b) * (I - I1) + i - I1];
        acc = fmaf(dy[static_cast<size_t>(b) * O + o], xv, acc);
      }
      dw[static_cast<size_t>(o) * I + i] = acc;
    }
  }
}

// One block per batch row: softmax cross-entropy over NT logits + lam * squared
// error of the two shift outputs; writes d(mean loss)/d out and the row loss.
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ out, const int* __restrict__ label,
                                              const float* __restrict__ target, int B, int NT, float lam,
                                              float* __restrict__ dout, float* __restrict__ loss) {
  const int b = blockIdx.x;
  const int stride = NT + 2;
  const float* o = out + static_cast<size_t>(b) * stride;
  __shared__ float red[256];
  float mx = -FLT_MAX;
  for (int k = threadIdx.x; k < NT; k += blockDim.x) mx = fmaxf(mx, o[k]);
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  mx = red[0];
  __syncthreads();
  float sum = 0.f;
  for (int k = threadIdx.x; k < NT; k += blockDim.x) sum += expf(o[k] - mx);
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  sum = red[0];
  const int lb = label[b];
  const bool lb_ok = lb >= 0 && lb < NT;  // an out-of-range label gives a NaN row loss
  const float invB = 1.f / B;
  float* d = dout + static_cast<size_t>(b) * stride;
  for (int k = threadIdx.x; k < NT; k += blockDim.x) d[k] = (expf(o[k] - mx) / sum - (k == lb ? 1.f : 0.f)) * invB;
  if (threadIdx.x < 2) d[NT + threadIdx.x] = 2.f * lam * (o[NT + threadIdx.x] - target[2 * b + threadIdx.x]) * invB;
  if (threadIdx.x == 0) {
    const float e0 = o[NT] - target[2 * b], e1 = o[NT + 1] - target[2 * b + 1];
    loss[b] = lb_ok ? -(o[lb] - mx - logf(sum)) + lam * (e0 * e0 + e1 * e1) : __int_as_float(0x7FC00000);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

// Order-preserving map of a float to a 32-bit unsigned key; NaN maps to 1 (below -inf),
// so that key 0 can mark entries already taken.
__device__ __forceinline__ unsigned int topk_key(float f) {
  if (f != f) return 1u;
  const unsigned int u = __float_as_uint(f);
  const unsigned int k = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return k < 2u ? 2u : k;
}

// One block per row: the k largest of NT logits (ties: lower index first), descending.
// Each candidate is the 64-bit key (value key << 32 | ~index); taken entries become 0,
// below every untaken one, so k <= NT distinct in-range indices are always produced.
__global__ void __launch_bounds__(256) k_topk(const float* __restrict__ out, int stride, int NT, int k,
                                              int* __restrict__ idx) {
  extern __shared__ unsigned long long sk[];  // NT keys
  __shared__ unsigned long long red[256];
  const int b = blockIdx.x;
  for (int j = threadIdx.x; j < NT; j += blockDim.x)
    sk[j] = (static_cast<unsigned long long>(topk_key(out[static_cast<size_t>(b) * stride + j])) << 32) |
            (0xFFFFFFFFu - static_cast<unsigned int>(j));
  __syncthreads();
  for (int t = 0; t < k; ++t) {
    unsigned long long best = 0ull;
    for (int j = threadIdx.x; j < NT; j += blockDim.x) best = sk[j] > best ? sk[j] : best;
    red[threadIdx.x] = best;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x + s] > red[threadIdx.x] ? red[threadIdx.x + s] : red[threadIdx.x];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int j = static_cast<int>(0xFFFFFFFFu - static_cast<unsigned int>(red[0] & 0xFFFFFFFFull));
      idx[static_cast<size_t>(b) * k + t] = j;
      sk[j] = 0ull;
    }
    __syncthreads();
  }
}

// conf[b] = softmax(out[b][0..NT)) summed over idx[b][0..K) (the shortlist's probability
// mass), or its largest value when idx is NULL.
__global__ void __launch_bounds__(256) k_confidence(const float* __restrict__ out, int stride, int NT,
                                                    const int* __restrict__ idx, int K, float* __restrict__ conf) {
  const int b = blockIdx.x;
  const float* o = out + static_cast<size_t>(b) * stride;
  __shared__ float red[256];
  float mx = -FLT_MAX;
  for (int k = threadIdx.x; k < NT; k += blockDim.x) mx = fmaxf(mx, o[k]);
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  mx = red[0];
  __syncthreads();
  float sum = 0.f;
  for (int k = threadIdx.x; k < NT; k += blockDim.x) sum += expf(o[k] - mx);
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  sum = red[0];
  __syncthreads();
  float part = 0.f;
  if (idx) {
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      const int j = idx[static_cast<size_t>(b) * K + k];
      if (j >= 0 && j < NT) part += expf(o[j] - mx);
    }
  } else if (threadIdx.x == 0) {
    part = 1.f;
  }
  red[threadIdx.x] = part;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) conf[b] = red[0] / sum;
}

// dst[r] = src[rows[r]]; a row index outside [0, n_src) yields a row of NaN.
__global__ void k_gather_rows(const float* __restrict__ src, long long n_src, const int* __restrict__ rows, long long n,
                              int row_elems, float* __restrict__ dst) {
  const long long total = n * row_elems;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = e / row_elems;
    const long long sr = rows[r];
    dst[e] = (sr >= 0 && sr < n_src) ? src[sr * row_elems + (e - r * row_elems)] : __int_as_float(0x7FC00000);
  }
}

// ---- rotation-equivariant template head ----
// X_ij(r) = Re sum_{m < Mh, |q| <= Qh} W_j(m, q) a_i(k_m; q) e^{-i q gamma_r}, gamma_r = 2 pi r / 2Q;
// logit_ij = alpha max_r X_ij(r) + beta_j (first maximising r). W is [NT][Mh][2Qh+1] complex
// (u = q + Qh), a is [B][M][2Q] complex with q stored at q mod 2Q.
constexpr int kEqTJ = 8;  // templates per block

__device__ __forceinline__ unsigned int eq_order_key(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ int mod_pos(long long x, int n) {
  const long long r = x % n;
  return static_cast<int>(r < 0 ? r + n : r);
}

// One block per (image, kEqTJ templates); 256 threads.
__global__ void __launch_bounds__(256) k_eqhead_fwd(const float2* __restrict__ a, int M, int two_Q,
                                                    const float2* __restrict__ W, const float* __restrict__ beta,
                                                    int NT, int Mh, int Qh, float alpha, float* __restrict__ out,
                                                    int out_stride, int accumulate, int* __restrict__ rstar) {
  extern __shared__ float2 eq_smem[];
  const int U = 2 * Qh + 1;
  float2* as = eq_smem;              // [Mh][U]
  float2* P = as + Mh * U;           // [kEqTJ][U]
  float2* tw = P + kEqTJ * U;        // [2Q]: e^{-i 2 pi t / 2Q}
  __shared__ unsigned long long red[8];
  const int i = blockIdx.x;
  const int j0 = blockIdx.y * kEqTJ;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < Mh * U; e += blockDim.x) {
    const int m = e / U, u = e - m * U;
    as[e] = a[(static_cast<size_t>(i) * M + m) * two_Q + mod_pos(u - Qh, two_Q)];
  }
  for (int t = tid; t < two_Q; t += blockDim.x) {
    float sn, cs;
    sincospif(2.f * static_cast<float>(t) / static_cast<float>(two_Q), &sn, &cs);
    tw[t] = make_float2(cs, -sn);
  }
  __syncthreads();
  for (int e = tid; e < kEqTJ * U; e += blockDim.x) {
    const int jl = e / U, u = e - jl * U;
    const int j = j0 + jl;
    float2 acc = make_float2(0.f, 0.f);
    if (j < NT) {
      const float2* wj = W + static_cast<size_t>(j) * Mh * U + u;
      for (int m = 0; m < Mh; ++m) {
        const float2 w = wj[static_cast<size_t>(m) * U];
        const float2 x = as[m * U + u];
        acc.x = fmaf(w.x, x.x, fmaf(-w.y, x.y, acc.x));
        acc.y = fmaf(w.x, x.y, fmaf(w.y, x.x, acc.y));
      }
    }
    P[e] = acc;
  }
  __syncthreads();
  for (int jl = 0; jl < kEqTJ; ++jl) {
    const int j = j0 + jl;
    if (j >= NT) break;  // uniform across the block
    unsigned long long best = 0ull;
    for (int r = tid; r < two_Q; r += blockDim.x) {
      int t = mod_pos(-static_cast<long long>(Qh) * r, two_Q);
      float x = 0.f;
      const float2* pj = P + jl * U;
      for (int u = 0; u < U; ++u) {
        const float2 pv = pj[u], e = tw[t];
        x = fmaf(pv.x, e.x, fmaf(-pv.y, e.y, x));
        t += r;
        if (t >= two_Q) t -= two_Q;
      }
      const unsigned long long k =
          (static_cast<unsigned long long>(eq_order_key(x)) << 32) | (0xFFFFFFFFu - static_cast<unsigned int>(r));
      best = k > best ? k : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
      best = v > best ? v : best;
    }
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (tid == 0) {
      unsigned long long b = red[0];
      for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) b = red[w] > b ? red[w] : b;
      const unsigned int hi = static_cast<unsigned int>(b >> 32);
      const float xmax = __uint_as_float((hi & 0x80000000u) ? (hi & 0x7FFFFFFFu) : ~hi);
      const int r = static_cast<int>(0xFFFFFFFFu - static_cast<unsigned int>(b & 0xFFFFFFFFull));
      float* o = out + static_cast<size_t>(i) * out_stride + j;
      const float v = fmaf(alpha, xmax, beta[j]);
      *o = accumulate ? *o + v : v;
      rstar[static_cast<size_t>(i) * NT + j] = r;
    }
    __syncthreads();
  }
}

// The same head with X_ij(r) for all r from one length-2Q FFT per pair: Z(q) = P_ij(q) on the
// band (zero elsewhere), X_ij(r) = Re sum_q Z(q) e^{-2 pi i q r / 2Q}. kEqIB images x kEqTJ
// templates per block; one warp per pair for the FFT (L = 2Q = 32 c, register FFT).
constexpr int kEqIB = 4;
template <int L>
__global__ void __launch_bounds__(256) k_eqhead_fwd_fft(const float2* __restrict__ a, int B, int M,
                                                        const float2* __restrict__ W, const float* __restrict__ beta,
                                                        int NT, int Mh, int Qh, float alpha, float* __restrict__ out,
                                                        int out_stride, int accumulate, int* __restrict__ rstar) {
  constexpr int c = L / 32;
  extern __shared__ float2 eq_smem[];
  const int U = 2 * Qh + 1;
  float2* tw = eq_smem;              // [L]: e^{-2 pi i t / L}
  float2* as = tw + L;               // [kEqIB][Mh][U]
  float2* P = as + kEqIB * Mh * U;   // [kEqIB * kEqTJ][U]
  const int i0 = blockIdx.x * kEqIB;
  const int j0 = blockIdx.y * kEqTJ;
  const int nib = min(kEqIB, B - i0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < L; t += blockDim.x) {
    float sn, cs;
    sincospif(2.f * static_cast<float>(t) / static_cast<float>(L), &sn, &cs);
    tw[t] = make_float2(cs, -sn);
  }
  for (int e = tid; e < kEqIB * Mh * U; e += blockDim.x) {
    const int ib = e / (Mh * U), rem = e - ib * Mh * U;
    const int m = rem / U, u = rem - m * U;
    as[e] = ib < nib ? a[(static_cast<size_t>(i0 + ib) * M + m) * L + mod_pos(u - Qh, L)] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int e = tid; e < kEqIB * kEqTJ * U; e += blockDim.x) {
    const int pr = e / U, u = e - pr * U;
    const int ib = pr / kEqTJ, jl = pr - ib * kEqTJ;
    const int j = j0 + jl;
    float2 acc = make_float2(0.f, 0.f);
    if (ib < nib && j < NT) {
      const float2* wj = W + static_cast<size_t>(j) * Mh * U + u;
      const float2* x = as + ib * Mh * U + u;
      for (int m = 0; m < Mh; ++m) {
        const float2 w = wj[static_cast<size_t>(m) * U];
        const float2 v = x[m * U];
        acc.x = fmaf(w.x, v.x, fmaf(-w.y, v.y, acc.x));
        acc.y = fmaf(w.x, v.y, fmaf(w.y, v.x, acc.y));
      }
    }
    P[e] = acc;
  }
  __syncthreads();
  const int br = __brev(lane) >> 27;
  for (int pr = warp; pr < kEqIB * kEqTJ; pr += blockDim.x >> 5) {
    const int ib = pr / kEqTJ, jl = pr - ib * kEqTJ;
    const int j = j0 + jl;
    if (ib >= nib || j >= NT) continue;  // uniform across the warp
    float2 v[c];
#pragma unroll
    for (int k = 0; k < c; ++k) {
      const int q = lane + 32 * k;
      const int u = (q < L / 2 ? q : q - L) + Qh;
      v[k] = (u >= 0 && u < U) ? P[pr * U + u] : make_float2(0.f, 0.f);
    }
    ftk::warp_fft<L>(v, tw);
    unsigned long long best = 0ull;
#pragma unroll
    for (int f2 = 0; f2 < c; ++f2) {
      const int r = f2 + c * br;
      const unsigned long long k =
          (static_cast<unsigned long long>(eq_order_key(v[f2].x)) << 32) | (0xFFFFFFFFu - static_cast<unsigned int>(r));
      best = k > best ? k : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, o);
      best = x > best ? x : best;
    }
    if (lane == 0) {
      const unsigned int hi = static_cast<unsigned int>(best >> 32);
      const float xmax = __uint_as_float((hi & 0x80000000u) ? (hi & 0x7FFFFFFFu) : ~hi);
      const int r = static_cast<int>(0xFFFFFFFFu - static_cast<unsigned int>(best & 0xFFFFFFFFull));
      const int i = i0 + ib;
      float* o = out + static_cast<size_t>(i) * out_stride + j;
      const float val = fmaf(alpha, xmax, beta[j]);
      *o = accumulate ? *o + val : val;
      rstar[static_cast<size_t>(i) * NT + j] = r;
    }
  }
}

template <int L>
cudaError_t launch_eqhead_fft(const float2* a, int B, int M, const float2* W, const float* beta, int NT, int Mh,
                              int Qh, float alpha, float* out, int out_stride, int accumulate, int* rstar,
                              cudaStream_t s, bool* done) {
  const int U = 2 * Qh + 1;
  const size_t smem = (static_cast<size_t>(L) + static_cast<size_t>(kEqIB) * Mh * U +
                       static_cast<size_t>(kEqIB) * kEqTJ * U) * sizeof(float2);
  *done = false;
  if (smem > 200 * 1024) return cudaSuccess;  // the direct kernel takes it
  cudaError_t e = cudaFuncSetAttribute(k_eqhead_fwd_fft<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((B + kEqIB - 1) / kEqIB, (NT + kEqTJ - 1) / kEqTJ);
  k_eqhead_fwd_fft<L><<<grid, 256, smem, s>>>(a, B, M, W, beta, NT, Mh, Qh, alpha, out, out_stride, accumulate, rstar);
  *done = true;
  return cudaGetLastError();
}

// One block per template j: dW_j(m, u) = alpha sum_i g_ij conj(a_i(k_m; q) e^{-i q gamma_{r*_ij}}),
// dbeta_j = sum_i g_ij, with g_ij = dout[i][j] (row stride out_stride).
__global__ void __launch_bounds__(256) k_eqhead_bwd(const float2* __restrict__ a, int B, int M, int two_Q,
                                                    const float* __restrict__ dout, int out_stride,
                                                    const int* __restrict__ rstar, int NT, int Mh, int Qh,
                                                    float alpha, float2* __restrict__ dW, float* __restrict__ dbeta) {
  extern __shared__ float2 eq_smem[];
  float2* tw = eq_smem;  // [2Q]
  const int U = 2 * Qh + 1;
  const int j = blockIdx.x;
  for (int t = threadIdx.x; t < two_Q; t += blockDim.x) {
    float sn, cs;
    sincospif(2.f * static_cast<float>(t) / static_cast<float>(two_Q), &sn, &cs);
    tw[t] = make_float2(cs, -sn);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < Mh * U; e += blockDim.x) {
    const int m = e / U, u = e - m * U;
    const int q = u - Qh;
    const int qs = mod_pos(q, two_Q);
    float2 acc = make_float2(0.f, 0.f);
    for (int i = 0; i < B; ++i) {
      const float g = dout[static_cast<size_t>(i) * out_stride + j];
      const int r = rstar[static_cast<size_t>(i) * NT + j];
      const float2 ph = tw[mod_pos(static_cast<long long>(q) * r, two_Q)];
      const float2 x = a[(static_cast<size_t>(i) * M + m) * two_Q + qs];
      // z = x * ph; acc += g * conj(z)
      const float zr = x.x * ph.x - x.y * ph.y, zi = x.x * ph.y + x.y * ph.x;
      acc.x = fmaf(g, zr, acc.x);
      acc.y = fmaf(-g, zi, acc.y);
    }
    dW[static_cast<size_t>(j) * Mh * U + e] = make_float2(alpha * acc.x, alpha * acc.y);
  }
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < B; ++i) s += dout[static_cast<size_t>(i) * out_stride + j];
    dbeta[j] = s;
  }
}

// dst[rows[r]] = src[r]; a row index outside [0, n_dst) is skipped.
__global__ void k_scatter_rows(const float* __restrict__ src, const int* __restrict__ rows, long long n, int row_elems,
                               float* __restrict__ dst, long long n_dst) {
  const long long total = n * row_elems;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = e / row_elems;
    const long long dr = rows[r];
    if (dr >= 0 && dr < n_dst) dst[dr * row_elems + (e - r * row_elems)] = src[e];
  }
}

// Template-head filters with a spectral weight shared by all templates:
// W[j][s] = rho[s] W0[j][s] (complex), s = (m, u) over the head's rings and angular band.
__global__ void k_scale_filters(const float2* __restrict__ W0, const float* __restrict__ rho, long long n, int S,
                                float2* __restrict__ W) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float r = rho[e % S];
    const float2 w = W0[e];
    W[e] = make_float2(r * w.x, r * w.y);
  }
}

// drho[s] = sum_j Re(dW[j][s]) Re(W0[j][s]) + Im(dW[j][s]) Im(W0[j][s]) (dW = dL/dRe W + i dL/dIm W):
// one thread per s, consecutive threads on consecutive s (coalesced over each template row).
__global__ void k_scale_filters_backward(const float2* __restrict__ W0, const float2* __restrict__ dW, int NT, int S,
                                         float* __restrict__ drho) {
  const int sidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (sidx >= S) return;
  float acc = 0.f;
  for (int j = 0; j < NT; ++j) {
    const size_t e = static_cast<size_t>(j) * S + sidx;
    const float2 d = dW[e], w = W0[e];
    acc = fmaf(d.x, w.x, fmaf(d.y, w.y, acc));
  }
  drho[sidx] = acc;
}

// out[b] = the shift nearest to center[b] in the max norm (ties: the lowest index), so
// that a window of any half-width >= 0 around out[b] holds at least that shift.
__global__ void k_snap_to_shifts(const float2* __restrict__ center, int B, const float2* __restrict__ shifts, int N,
                                 float2* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float2 c = center[b];
  float best = INFINITY;
  int bs = 0;
  for (int s = 0; s < N; ++s) {
    const float2 v = shifts[s];
    const float d = fmaxf(fabsf(v.x - c.x), fabsf(v.y - c.y));
    if (d < best) {
      best = d;
      bs = s;
    }
  }
  out[b] = shifts[bs];
}

// Appends every b with val[b] < thr to rows (in no particular order); *count ends as their number.
__global__ void k_select_below(const float* __restrict__ val, long long n, float thr, int* __restrict__ rows,
                               int* __restrict__ count) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const bool take = val[e] < thr;
    const unsigned mask = __ballot_sync(__activemask(), take);
    if (!take) continue;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    rows[base + __popc(mask & ((1u << lane) - 1u))] = static_cast<int>(e);
  }
}

unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 148LL * 64) g = 148LL * 64;
  return static_cast<unsigned>(g < 1 ? 1 : g);
}

cudaStream_t st(void* s) { return static_cast<cudaStream_t>(s); }

ftk_status launched() { return cudaGetLastError() == cudaSuccess ? FTK_OK : FTK_ERR_CUDA; }

}  // namespace

extern "C" {

ftk_status ftk_nn_features(const float* d_coeffs, int B, int M, int two_Q, float eps_f, float* d_x0, float* d_lin,
                           void* stream) {
  if (B < 0 || M < 1 || two_Q < 4 || (two_Q & 1) || !(eps_f > 0)) return FTK_ERR_ARG;
  if (B == 0) return FTK_OK;
  if (!d_coeffs || !d_x0 || !d_lin) return FTK_ERR_ARG;
  const long long n = static_cast<long long>(B) * M * (two_Q / 2);
  k_nn_features<<<grid_for(n), 256, 0, st(stream)>>>(reinterpret_cast<const float2*>(d_coeffs), B, M, two_Q, eps_f,
                                                      d_x0, d_lin);
  return launched();
}

ftk_status ftk_nn_conv3x3(const float* d_x, const float* d_w, const float* d_b, float* d_y, int B, int Ci, int Co,
                          int H, int W, int relu, void* stream) {
  if (B < 0 || Ci < 1 || Co < 1 || H < 1 || W < 1 || !d_x || !d_w || !d_b || !d_y) return FTK_ERR_ARG;
  const long long n = static_cast<long long>(B) * Co * H * W;
  if (n == 0) return FTK_OK;
  k_conv3x3<<<grid_for(n), 256, 0, st(stream)>>>(d_x, d_w, d_b, d_y, B, Ci, Co, H, W, relu);
  return launched();
}

ftk_status ftk_nn_conv3x3_backward(const float* d_x, const float* d_w, const float* d_dz, float* d_dx, float* d_dw,
                                   float* d_db, int B, int Ci, int Co, int H, int W, void* stream) {
  if (B < 1 || Ci < 1 || Co < 1 || H < 1 || W < 1 || !d_x || !d_w || !d_dz || !d_dw || !d_db) return FTK_ERR_ARG;
  if (d_dx) {
    const long long n = static_cast<long long>(B) * Ci * H * W;
    k_conv3x3_bwd_data<<<grid_for(n), 256, 0, st(stream)>>>(d_w, d_dz, d_dx, B, Ci, Co, H, W);
    if (cudaGetLastError() != cudaSuccess) return FTK_ERR_CUDA;
  }
  k_conv3x3_bwd_weight<<<Co * Ci, 256, 0, st(stream)>>>(d_x, d_dz, d_dw, d_db, B, Ci, Co, H, W);
  return launched();
}

ftk_status ftk_nn_relu_backward(const float* d_y, float* d_dy, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!d_y || !d_dy))) return FTK_ERR_ARG;
  if (n == 0) return FTK_OK;
  k_relu_bwd<<<grid_for(n), 256, 0, st(stream)>>>(d_y, d_dy, n);
  return launched();
}

ftk_status ftk_nn_pool2(const float* d_x, float* d_y, long long BC, int H, int W, void* stream) {
  if (BC < 0 || H < 2 || W < 2 || (H & 1) || (W & 1) || !d_x || !d_y) return FTK_ERR_ARG;
  k_pool2<<<grid_for(BC * H * W / 4), 256, 0, st(stream)>>>(d_x, d_y, BC, H, W);
  return launched();
}

ftk_status ftk_nn_pool2_backward(const float* d_dy, float* d_dx, long long BC, int H, int W, void* stream) {
  if (BC < 0 || H < 2 || W < 2 || (H & 1) || (W & 1) || !d_dy || !d_dx) return FTK_ERR_ARG;
  k_pool2_bwd<<<grid_for(BC * H * W), 256, 0, st(stream)>>>(d_dy, d_dx, BC, H, W);
  return launched();
}

ftk_status ftk_nn_gap(const float* d_x, float* d_y, long long BC, int HW, void* stream) {
  if (BC < 0 || HW < 1 || !d_x || !d_y) return FTK_ERR_ARG;
  k_gap<<<grid_for(BC), 256, 0, st(stream)>>>(d_x, d_y, BC, HW);
  return launched();
}

ftk_status ftk_nn_gap_backward(const float* d_dy, float* d_dx, long long BC, int HW, void* stream) {
  if (BC < 0 || HW < 1 || !d_dy || !d_dx) return FTK_ERR_ARG;
  k_gap_bwd<<<grid_for(BC * HW), 256, 0, st(stream)>>>(d_dy, d_dx, BC, HW);
  return launched();
}

ftk_status ftk_nn_linear(const float* d_x1, const float* d_x2, int I1, const float* d_w, const float* d_b, float* d_y,
                         int B, int I, int O, int relu, void* stream) {
  if (B < 0 || I < 1 || O < 1 || I1 < 1 || I1 > I || (I1 < I && !d_x2) || !d_x1 || !d_w || !d_b || !d_y)
    return FTK_ERR_ARG;
  k_linear<<<grid_for(static_cast<long long>(B) * O), 256, 0, st(stream)>>>(d_x1, I1 < I ? d_x2 : nullptr, I1, d_w,
                                                                              d_b, d_y, B, I, O, relu);
  return launched();
}

ftk_status ftk_nn_linear_backward(const float* d_x1, const float* d_x2, int I1, const float* d_w, const float* d_dy,
                                  float* d_dx1, float* d_dw, float* d_db, int B, int I, int O, void* stream) {
  if (B < 1 || I < 1 || O < 1 || I1 < 1 || I1 > I || (I1 < I && !d_x2) || !d_x1 || !d_w || !d_dy || !d_dw || !d_db)
    return FTK_ERR_ARG;
  if (d_dx1) {
    k_linear_bwd_data<<<grid_for(static_cast<long long>(B) * I1), 256, 0, st(stream)>>>(d_dy, d_w, d_dx1, B, I, O, I1);
    if (cudaGetLastError() != cudaSuccess) return FTK_ERR_CUDA;
  }
  k_linear_bwd_weight<<<grid_for(static_cast<long long>(O) * (I + 1)), 256, 0, st(stream)>>>(
      d_x1, I1 < I ? d_x2 : nullptr, I1, d_dy, d_dw, d_db, B, I, O);
  return launched();
}

ftk_status ftk_nn_loss(const float* d_out, const int* d_label, const float* d_target, int B, int NT, float lam,
                       float* d_dout, float* d_loss, void* stream) {
  if (B < 1 || NT < 1 || !d_out || !d_label || !d_target || !d_dout || !d_loss) return FTK_ERR_ARG;
  k_loss<<<B, 256, 0, st(stream)>>>(d_out, d_label, d_target, B, NT, lam, d_dout, d_loss);
  return launched();
}

ftk_status ftk_nn_adam(float* d_p, const float* d_g, float* d_m, float* d_v, long long n, float lr, float b1, float b2,
                       float eps, int t, void* stream) {
  if (n < 0 || t < 1 || !d_p || !d_g || !d_m || !d_v) return FTK_ERR_ARG;
  const float c1 = 1.f - powf(b1, static_cast<float>(t)), c2 = 1.f - powf(b2, static_cast<float>(t));
  k_adam<<<grid_for(n), 256, 0, st(stream)>>>(d_p, d_g, d_m, d_v, n, lr, b1, b2, eps, c1, c2);
  return launched();
}

ftk_status ftk_nn_topk(const float* d_out, int B, int stride, int NT, int k, int* d_idx, void* stream) {
  if (B < 0 || NT < 1 || k < 1 || k > NT || stride < NT || !d_out || !d_idx) return FTK_ERR_ARG;
  if (B == 0) return FTK_OK;
  const size_t smem = static_cast<size_t>(NT) * sizeof(unsigned long long);
  if (smem > 160 * 1024) return FTK_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return FTK_ERR_CUDA;
  k_topk<<<B, 256, smem, st(stream)>>>(d_out, stride, NT, k, d_idx);
  return launched();
}

ftk_status ftk_nn_confidence(const float* d_out, int B, int stride, int NT, const int* d_idx, int K, float* d_conf,
                             void* stream) {
  if (B < 0 || NT < 1 || stride < NT || !d_out || !d_conf || (d_idx && (K < 1 || K > NT))) return FTK_ERR_ARG;
  if (B == 0) return FTK_OK;
  k_confidence<<<B, 256, 0, st(stream)>>>(d_out, stride, NT, d_idx, K, d_conf);
  return launched();
}

ftk_status ftk_nn_eqhead(const float* d_a, int B, int M, int two_Q, const float* d_W, const float* d_beta, int NT,
                         int Mh, int Qh, float alpha, float* d_out, int out_stride, int accumulate, int* d_rstar,
                         void* stream) {
  if (B < 0 || M < 1 || two_Q < 2 || NT < 1 || Mh < 1 || Mh > M || Qh < 0 || 2 * Qh + 1 > two_Q ||
      out_stride < NT)
    return FTK_ERR_ARG;
  if (B == 0) return FTK_OK;
  if (!d_a || !d_W || !d_beta || !d_out || !d_rstar) return FTK_ERR_ARG;
  if ((NT + kEqTJ - 1) / kEqTJ > 65535) return FTK_ERR_UNSUPPORTED;
  {
    const float2* a2 = reinterpret_cast<const float2*>(d_a);
    const float2* W2 = reinterpret_cast<const float2*>(d_W);
    bool done = false;
    cudaError_t e = cudaSuccess;
    switch (two_Q) {
      case 96: e = launch_eqhead_fft<96>(a2, B, M, W2, d_beta, NT, Mh, Qh, alpha, d_out, out_stride, accumulate, d_rstar, st(stream), &done); break;
      case 192: e = launch_eqhead_fft<192>(a2, B, M, W2, d_beta, NT, Mh, Qh, alpha, d_out, out_stride, accumulate, d_rstar, st(stream), &done); break;
      case 288: e = launch_eqhead_fft<288>(a2, B, M, W2, d_beta, NT, Mh, Qh, alpha, d_out, out_stride, accumulate, d_rstar, st(stream), &done); break;
      case 384: e = launch_eqhead_fft<384>(a2, B, M, W2, d_beta, NT, Mh, Qh, alpha, d_out, out_stride, accumulate, d_rstar, st(stream), &done); break;
      case 576: e = launch_eqhead_fft<576>(a2, B, M, W2, d_beta, NT, Mh, Qh, alpha, d_out, out_stride, accumulate, d_rstar, st(stream), &done); break;
      default: break;
    }
    if (e != cudaSuccess) return FTK_ERR_CUDA;
    if (done) return FTK_OK;
  }
  const int U = 2 * Qh + 1;
  const size_t smem = (static_cast<size_t>(Mh) * U + static_cast<size_t>(kEqTJ) * U + two_Q) * sizeof(float2);
  if (smem > 200 * 1024) return FTK_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_eqhead_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
      cudaSuccess)
    return FTK_ERR_CUDA;
  dim3 grid(B, (NT + kEqTJ - 1) / kEqTJ);
  k_eqhead_fwd<<<grid, 256, smem, st(stream)>>>(reinterpret_cast<const float2*>(d_a), M, two_Q,
                                                reinterpret_cast<const float2*>(d_W), d_beta, NT, Mh, Qh, alpha,
                                                d_out, out_stride, accumulate, d_rstar);
  return launched();
}

ftk_status ftk_nn_eqhead_backward(const float* d_a, int B, int M, int two_Q, const float* d_dout, int out_stride,
                                  const int* d_rstar, int NT, int Mh, int Qh, float alpha, float* d_dW, float* d_dbeta,
                                  void* stream) {
  if (B < 1 || M < 1 || two_Q < 2 || NT < 1 || Mh < 1 || Mh > M || Qh < 0 || 2 * Qh + 1 > two_Q ||
      out_stride < NT || !d_a || !d_dout || !d_rstar || !d_dW || !d_dbeta)
    return FTK_ERR_ARG;
  const size_t smem = static_cast<size_t>(two_Q) * sizeof(float2);
  if (smem > 48 * 1024) return FTK_ERR_UNSUPPORTED;
  k_eqhead_bwd<<<NT, 256, smem, st(stream)>>>(reinterpret_cast<const float2*>(d_a), B, M, two_Q, d_dout, out_stride,
                                              d_rstar, NT, Mh, Qh, alpha, reinterpret_cast<float2*>(d_dW), d_dbeta);
  return launched();
}

ftk_status ftk_scatter_rows(const float* d_src, const int* d_rows, long long n, int row_elems, float* d_dst,
                            long long n_dst, void* stream) {
  if (n < 0 || n_dst < 0 || row_elems < 1 || (n > 0 && (!d_src || !d_rows || !d_dst))) return FTK_ERR_ARG;
  if (n == 0) return FTK_OK;
  k_scatter_rows<<<grid_for(n * row_elems), 256, 0, st(stream)>>>(d_src, d_rows, n, row_elems, d_dst, n_dst);
  return launched();
}

ftk_status ftk_nn_scale_filters(const float* d_W0, const float* d_rho, int NT, int S, float* d_W, void* stream) {
  if (NT < 1 || S < 1 || !d_W0 || !d_rho || !d_W) return FTK_ERR_ARG;
  const long long n = static_cast<long long>(NT) * S;
  k_scale_filters<<<grid_for(n), 256, 0, st(stream)>>>(reinterpret_cast<const float2*>(d_W0), d_rho, n, S,
                                                     reinterpret_cast<float2*>(d_W));
  return launched();
}

ftk_status ftk_nn_scale_filters_backward(const float* d_W0, const float* d_dW, int NT, int S, float* d_drho,
                                         void* stream) {
  if (NT < 1 || S < 1 || !d_W0 || !d_dW || !d_drho) return FTK_ERR_ARG;
  k_scale_filters_backward<<<(S + 255) / 256, 256, 0, st(stream)>>>(reinterpret_cast<const float2*>(d_W0),
                                                                   reinterpret_cast<const float2*>(d_dW), NT, S,
                                                                   d_drho);
  return launched();
}

ftk_status ftk_nn_snap_to_shifts(const float* d_center, int B, const float* d_shifts, int N, float* d_out,
                                 void* stream) {
  if (B < 0 || N < 1 || (B > 0 && (!d_center || !d_shifts || !d_out))) return FTK_ERR_ARG;
  if (B == 0) return FTK_OK;
  k_snap_to_shifts<<<(B + 255) / 256, 256, 0, st(stream)>>>(reinterpret_cast<const float2*>(d_center), B,
                                                           reinterpret_cast<const float2*>(d_shifts), N,
                                                           reinterpret_cast<float2*>(d_out));
  return launched();
}

ftk_status ftk_select_below(const float* d_val, long long n, float thr, int* d_rows, int* d_count, void* stream) {
  if (n < 0 || n > 2147483647LL || !d_count || (n > 0 && (!d_val || !d_rows))) return FTK_ERR_ARG;
  if (cudaMemsetAsync(d_count, 0, sizeof(int), st(stream)) != cudaSuccess) return FTK_ERR_CUDA;
  if (n == 0) return FTK_OK;
  k_select_below<<<grid_for(n), 256, 0, st(stream)>>>(d_val, n, thr, d_rows, d_count);
  return launched();
}

ftk_status ftk_gather_rows(const float* d_src, long long n_src, const int* d_rows, long long n, int row_elems,
                           float* d_dst, void* stream) {
  if (n < 0 || n_src < 0 || row_elems < 1 || (n > 0 && (!d_src || !d_rows || !d_dst))) return FTK_ERR_ARG;
  if (n == 0) return FTK_OK;
  k_gather_rows<<<grid_for(n * row_elems), 256, 0, st(stream)>>>(d_src, n_src, d_rows, n, row_elems, d_dst);
  return launched();
}

}  // extern "C"
