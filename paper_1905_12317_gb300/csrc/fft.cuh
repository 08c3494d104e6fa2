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

// ---- compile-time length: divisions by the radix and stride fold into
// multiply-shift sequences and the radix schedule unrolls. Transform t lives at
// buf + t * PS (PS >= L; padding spreads shared-memory banks).
template <int L, int PS, int R, int Ns>
__device__ __forceinline__ void stockham_pass_c(const float2* __restrict__ src, float2* __restrict__ dst, int T,
                                                const float2* __restrict__ tw) {
  constexpr int nb = L / R;
  constexpr int step = L / (Ns * R);
  for (int idx = threadIdx.x; idx < T * nb; idx += blockDim.x) {
    const int t = idx / nb;
    const int j = idx - t * nb;
    const int k = j % Ns;
    const float2* s = src + t * PS;
    float2* d = dst + t * PS;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = s[j + r * nb];
      if (r) v[r] = cmul(v[r], tw[k * r * step]);
    }
    dft_small<R>(v);
    const int o = (j / Ns) * (Ns * R) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[o + r * Ns] = v[r];
  }
}

// Radix order 4, 2, 3 (as make_fft_schedule).
template <int L, int PS, int Ns, int Rem>
struct StockhamC {
  static __device__ __forceinline__ float2* run(float2* a, float2* b, int T, const float2* tw) {
    constexpr int R = (Rem % 4 == 0) ? 4 : ((Rem % 2 == 0) ? 2 : 3);
    stockham_pass_c<L, PS, R, Ns>(a, b, T, tw);
    __syncthreads();
    return StockhamC<L, PS, Ns * R, Rem / R>::run(b, a, T, tw);
  }
};
template <int L, int PS, int Ns>
struct StockhamC<L, PS, Ns, 1> {
  static __device__ __forceinline__ float2* run(float2* a, float2*, int, const float2*) { return a; }
};

template <int L, int PS>
__device__ __forceinline__ float2* stockham_fft_c(float2* buf0, float2* buf1, int T, const float2* tw) {
  return StockhamC<L, PS, 1, L>::run(buf0, buf1, T, tw);
}

// ---- register FFT: one warp per length-L transform, L = 32 c ----------------
// Lane t holds x[t + 32 k], k < c. With n = t + 32 k and output f = f2 + c f1:
//   Y_t[f2] = sum_k x[t + 32 k] w_c^{k f2}            (DFT-c in registers)
//   Y_t[f2] *= w_L^{t f2}                             (twiddle)
//   X[f2 + c f1] = sum_t Y_t[f2] w_32^{t f1}          (DFT-32 across lanes)
// tw[e] = exp(-2 pi i e / L); w_N^e = tw[(e L / N) mod L].

// In-register DFT of compile-time size N (N = 1, 2, 3, 4 direct; otherwise split
// N = R M with R = 3 (or 2) and recurse): v[k] <- sum_n v[n] w_N^{n k}.
template <int N, int L>
struct RegDft {
  static __device__ __forceinline__ void run(float2* v, const float2* __restrict__ tw) {
    if constexpr (N == 1) {
    } else if constexpr (N == 2 || N == 3 || N == 4) {
      dft_small<N>(v);
    } else {
      constexpr int R = (N % 3 == 0) ? 3 : ((N % 4 == 0) ? 4 : 2);
      constexpr int Mm = N / R;
      // decimation in time: E_r = DFT_M(v[r], v[R + r], ...)
      float2 e[R][Mm];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int m = 0; m < Mm; ++m) e[r][m] = v[m * R + r];
#pragma unroll
      for (int r = 0; r < R; ++r) RegDft<Mm, L>::run(e[r], tw);
      // X[k' + M q] = sum_r (w_N^{r k'} E_r[k']) w_R^{r q}
#pragma unroll
      for (int kp = 0; kp < Mm; ++kp) {
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = (r * kp) ? cmul(e[r][kp], tw[(r * kp * (L / N)) % L]) : e[r][kp];
        dft_small<R>(u);
#pragma unroll
        for (int q = 0; q < R; ++q) v[kp + Mm * q] = u[q];
      }
    }
  }
};

// Full transform of the warp's 32 c values; on return lane t holds
// X[f2 + c * bitrev5(t)] in v[f2].
template <int L>
__device__ __forceinline__ void warp_fft(float2* v, const float2* __restrict__ tw) {
  constexpr int c = L / 32;
  const int t = threadIdx.x & 31;
  RegDft<c, L>::run(v, tw);
#pragma unroll
  for (int f2 = 1; f2 < c; ++f2) v[f2] = cmul(v[f2], tw[(t * f2) % L]);
  // DFT-32 across lanes, decimation in frequency (bit-reversed output)
  // Branch-free butterfly: lower lane v + p, upper lane (p - v) w, written as
  // (p + sgn v) w' with sgn = +1 / -1 and w' = 1 / w for the lower / upper lane.
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const bool upper = (t & d) != 0;
    const float sgn = upper ? -1.f : 1.f;
    const float2 w = upper ? tw[((t & (d - 1)) * (16 / d) * c) % L] : make_float2(1.f, 0.f);
#pragma unroll
    for (int f2 = 0; f2 < c; ++f2) {
      float2 p;
      p.x = __shfl_xor_sync(0xFFFFFFFFu, v[f2].x, d);
      p.y = __shfl_xor_sync(0xFFFFFFFFu, v[f2].y, d);
      const float2 s = make_float2(fmaf(sgn, v[f2].x, p.x), fmaf(sgn, v[f2].y, p.y));
      v[f2] = cmul(s, w);
    }
  }
}

// Transform of length L by a group of G lanes (G a power of two dividing 32, L = G c):
// on entry lane t of the group holds x[t + G k] in v[k]; on return it holds
// X[f2 + c * bitrev(t)] in v[f2] (bitrev over log2 G bits). warp_fft is G = 32.
// Fewer lanes per transform mean more values per lane and fewer shuffle stages
// (log2 G butterflies across lanes).
template <int L, int G>
__device__ __forceinline__ void group_fft(float2* v, const float2* __restrict__ tw) {
  constexpr int c = L / G;
  static_assert(G * c == L && (G & (G - 1)) == 0 && G <= 32, "L = G c, G a power of two <= 32");
  const int t = threadIdx.x & (G - 1);
  RegDft<c, L>::run(v, tw);
#pragma unroll
  for (int f2 = 1; f2 < c; ++f2) v[f2] = cmul(v[f2], tw[(t * f2) % L]);
#pragma unroll
  for (int d = G / 2; d >= 1; d >>= 1) {
    const bool upper = (t & d) != 0;
    const float sgn = upper ? -1.f : 1.f;
    const float2 w = upper ? tw[((t & (d - 1)) * (G / 2 / d) * c) % L] : make_float2(1.f, 0.f);
#pragma unroll
    for (int f2 = 0; f2 < c; ++f2) {
      float2 p;
      p.x = __shfl_xor_sync(0xFFFFFFFFu, v[f2].x, d);
      p.y = __shfl_xor_sync(0xFFFFFFFFu, v[f2].y, d);
      const float2 s = make_float2(fmaf(sgn, v[f2].x, p.x), fmaf(sgn, v[f2].y, p.y));
      v[f2] = cmul(s, w);
    }
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

// ---- DFTs in registers, forward sign; w_N^m = tw[m * ts] with tw[t] = w_L^t ----
template <int N>
__device__ __forceinline__ void dft_reg(float2* x, const float2* tw, int ts);

// N = P R: input n = R a + b, output k = c + P d.
template <int P, int R>
__device__ __forceinline__ void ct_pass(float2* x, const float2* tw, int ts) {
  float2 u[R][P];
#pragma unroll
  for (int b = 0; b < R; ++b) {
    float2 t[P];
#pragma unroll
    for (int a = 0; a < P; ++a) t[a] = x[R * a + b];
    dft_reg<P>(t, tw, ts * R);
#pragma unroll
    for (int c = 0; c < P; ++c) u[b][c] = (b && c) ? cmul(t[c], tw[b * c * ts]) : t[c];
  }
#pragma unroll
  for (int c = 0; c < P; ++c) {
    float2 t[R];
#pragma unroll
    for (int b = 0; b < R; ++b) t[b] = u[b][c];
    dft_reg<R>(t, tw, ts * P);
#pragma unroll
    for (int d = 0; d < R; ++d) x[c + P * d] = t[d];
  }
}

template <int N>
__device__ __forceinline__ void dft_reg(float2* x, const float2* tw, int ts) {
  if constexpr (N == 2 || N == 3 || N == 4) {
    dft_small<N>(x);
  } else if constexpr (N == 8) {
    ct_pass<4, 2>(x, tw, ts);
  } else if constexpr (N == 12) {
    ct_pass<4, 3>(x, tw, ts);
  } else if constexpr (N == 16) {
    ct_pass<4, 4>(x, tw, ts);
  } else if constexpr (N == 24) {
    ct_pass<8, 3>(x, tw, ts);
  } else if constexpr (N == 32) {
    ct_pass<4, 8>(x, tw, ts);
  } else {
    static_assert(N < 0, "unsupported DFT length");
  }
}

}  // namespace ftk
