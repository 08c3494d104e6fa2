// Mixed-radix (2, 3, 4) Stockham FFT on shared memory, forward sign
// exp(-2 pi i t r / L). Used for the ring DFT of eq. (aqkcalc) and for Step 2 of
// eq. (fbk3) (the DFT over q that yields every rotation gamma_r = pi r / Q).
#pragma once

#include <cuda_runtime.h>

namespace ftk {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <int R>
__device__ __forceinline__ void dft_small(float2* v) {
  if constexpr (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const float2 a = v[0], b = v[1], c = v[2], d = v[3];
    const float2 ac = cadd(a, c), amc = csub(a, c), bd = cadd(b, d), bmd = csub(b, d);
    v[0] = cadd(ac, bd);
    v[2] = csub(ac, bd);
    // X1 = (a - c) - i (b - d), X3 = (a - c) + i (b - d)
    v[1] = make_float2(amc.x + bmd.y, amc.y - bmd.x);
    v[3] = make_float2(amc.x - bmd.y, amc.y + bmd.x);
  } else if constexpr (R == 3) {
    // omega = exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2
    const float s3 = 0.86602540378443864676f;
    const float2 a = v[0], b = v[1], c = v[2];
    const float2 t = cadd(b, c), d = csub(b, c);
    v[0] = cadd(a, t);
    const float2 m = make_float2(a.x - 0.5f * t.x, a.y - 0.5f * t.y);
    // -i s3 (b - c) = (s3 d.y, -s3 d.x)
    v[1] = make_float2(m.x + s3 * d.y, m.y - s3 * d.x);
    v[2] = make_float2(m.x - s3 * d.y, m.y + s3 * d.x);
  }
}

// One Stockham pass of radix R over T transforms of length L stored
// contiguously in src; writes dst. tw[t] = exp(-2 pi i t / L).
template <int R>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ src, float2* __restrict__ dst,
                                              int T, int L, int Ns, const float2* __restrict__ tw) {
  const int nb = L / R;
  const int step = L / (Ns * R);
  for (int idx = threadIdx.x; idx < T * nb; idx += blockDim.x) {
    const int t = idx / nb;
    const int j = idx - t * nb;
    const int k = j % Ns;
    const float2* s = src + t * L;
    float2* d = dst + t * L;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = s[j + r * nb];
      if (r) v[r] = cmul(v[r], tw[k * r * step]);
    }
    dft_small<R>(v);
    const int o = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[o + r * Ns] = v[r];
  }
}

// Full transform; returns the buffer that holds the result (buf0 or buf1).
__device__ __forceinline__ float2* stockham_fft(float2* buf0, float2* buf1, int T, int L, const int* radix,
                                               int nradix, const float2* tw) {
  int Ns = 1;
  float2* a = buf0;
  float2* b = buf1;
  for (int ps = 0; ps < nradix; ++ps) {
    const int R = radix[ps];
    if (R == 4) stockham_pass<4>(a, b, T, L, Ns, tw);
    else if (R == 2) stockham_pass<2>(a, b, T, L, Ns, tw);
    else stockham_pass<3>(a, b, T, L, Ns, tw);
    __syncthreads();
    float2* c = a;
    a = b;
    b = c;
    Ns *= R;
  }
  return a;
}

}  // namespace ftk
