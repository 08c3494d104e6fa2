// FP32 SIMT pair engine: Steps 1 and 3 of eq. (fbk3) (Section 4.5) and the
// per-image best-pose epilogue. Step 2 (DFT over q) is launch_fft_rows.
//
// Only the orders l >= 0 are evaluated. For real images
// a(k; -q) = (-1)^q conj a(k; q), and the SVD of J_{-l} = (-1)^l J_l gives
// G_eta(k; -l) = G_eta(k; l), Y_eta(delta; -l) = (-1)^l conj Y_eta(delta; l), hence
// Zhat_{eta,-l}(q) = (-1)^l conj Zhat_{eta,l}(-q), Y_{-l} Z_{-l} = conj(Y_l Z_l), and
// X = Re sum_zeta Y_zeta Z_zeta = Re sum_{l >= 0} c_l Y_zeta Z_zeta with c_0 = 1,
// c_l = 2 (l > 0). The factor c_l is folded into the plan's Y table.
#include "fft.cuh"
#include "ftk_internal.h"

namespace ftk {

namespace {

constexpr int kS1Threads = 128;
constexpr int kS1TJ = 8;  // templates per thread

// Step 1: Zhat_zeta(q) = sum_m [2 pi w_m G_zeta(k_m)] a_i(k_m; q - l_zeta) conj b_j(k_m; q),
// for every (zeta, q) of one image i and kS1TJ templates j. Output [pair][zeta][q].
// With `list`, image i's templates are b[list[i * nj + jj]] (a per-image shortlist).
__global__ void __launch_bounds__(kS1Threads) k_step1_simt(
    const float2* __restrict__ a, const float2* __restrict__ b, int nj, const float* __restrict__ G,
    const int* __restrict__ lz, int Hh, int M, int two_Q, float2* __restrict__ zhat, const int* __restrict__ list) {
  const int e = blockIdx.x * kS1Threads + threadIdx.x;
  if (e >= Hh * two_Q) return;
  const int i = blockIdx.y;
  const int j0 = blockIdx.z * kS1TJ;
  const int zeta = e / two_Q;
  const int q = e - zeta * two_Q;
  int qa = q - lz[zeta];
  qa += (qa < 0) ? two_Q : 0;
  const float2* ai = a + static_cast<size_t>(i) * M * two_Q;
  const float* g = G + static_cast<size_t>(zeta) * M;
  const int ntj = min(kS1TJ, nj - j0);
  float2 acc[kS1TJ];
#pragma unroll
  for (int t = 0; t < kS1TJ; ++t) acc[t] = make_float2(0.f, 0.f);
  for (int m = 0; m < M; ++m) {
    const float gm = __ldg(g + m);
    const float2 av0 = __ldg(ai + m * two_Q + qa);
    const float2 av = make_float2(gm * av0.x, gm * av0.y);
#pragma unroll
    for (int t = 0; t < kS1TJ; ++t) {
      if (t < ntj) {
        const int jr = list ? __ldg(list + static_cast<size_t>(i) * nj + j0 + t) : j0 + t;
        const float2 bv = __ldg(b + (static_cast<size_t>(jr) * M + m) * two_Q + q);
        // av * conj(bv)
        acc[t].x = fmaf(av.x, bv.x, fmaf(av.y, bv.y, acc[t].x));
        acc[t].y = fmaf(av.y, bv.x, fmaf(-av.x, bv.y, acc[t].y));
      }
    }
  }
#pragma unroll
  for (int t = 0; t < kS1TJ; ++t) {
    if (t < ntj) zhat[(static_cast<size_t>(i) * nj + j0 + t) * Hh * two_Q + e] = acc[t];
  }
}

// Step 1 for per-image template lists, written in the layout of the tensor-core Steps 2-3:
// Zhat [pair][q][zeta] with row stride Hs = Hh rounded up to even, pair = i * nj + jj and
// template list[i * nj + jj]. Consecutive threads take consecutive zeta of one q, so the
// stores are coalesced, b(k_m; q) is a broadcast, and G is read from a transposed copy in
// shared memory ([m][zeta], conflict-free); the a(k_m; q - l_zeta) reads gather within one
// image row.
constexpr int kL1TJ = 8;  // templates per thread
__global__ void __launch_bounds__(kS1Threads) k_step1_list_tc(
    const float2* __restrict__ a, const float2* __restrict__ b, int nj, const float* __restrict__ G,
    const int* __restrict__ lz, int Hh, int M, int two_Q, float2* __restrict__ zhat, const int* __restrict__ list) {
  extern __shared__ float gt[];  // [M][Hh]
  for (int t = threadIdx.x; t < M * Hh; t += blockDim.x) {
    const int m = t / Hh, z = t - m * Hh;
    gt[t] = G[static_cast<size_t>(z) * M + m];
  }
  __syncthreads();
  const int e = blockIdx.x * kS1Threads + threadIdx.x;
  if (e >= Hh * two_Q) return;
  const int i = blockIdx.y;
  const int j0 = blockIdx.z * kL1TJ;
  const int q = e / Hh;
  const int zeta = e - q * Hh;
  const int Hs = (Hh + 1) & ~1;
  int qa = q - lz[zeta];
  qa += (qa < 0) ? two_Q : 0;
  const float2* ai = a + static_cast<size_t>(i) * M * two_Q;
  const int ntj = min(kL1TJ, nj - j0);
  const float2* bp[kL1TJ];
#pragma unroll
  for (int t = 0; t < kL1TJ; ++t)
    bp[t] = b + static_cast<size_t>(t < ntj ? __ldg(list + static_cast<size_t>(i) * nj + j0 + t) : 0) * M * two_Q + q;
  float2 acc[kL1TJ];
#pragma unroll
  for (int t = 0; t < kL1TJ; ++t) acc[t] = make_float2(0.f, 0.f);
  for (int m = 0; m < M; ++m) {
    const float gm = gt[m * Hh + zeta];
    const float2 av0 = __ldg(ai + m * two_Q + qa);
    const float2 av = make_float2(gm * av0.x, gm * av0.y);
#pragma unroll
    for (int t = 0; t < kL1TJ; ++t) {
      if (t < ntj) {
        const float2 bv = __ldg(bp[t] + static_cast<size_t>(m) * two_Q);
        acc[t].x = fmaf(av.x, bv.x, fmaf(av.y, bv.y, acc[t].x));
        acc[t].y = fmaf(av.y, bv.x, fmaf(-av.x, bv.y, acc[t].y));
      }
    }
  }
#pragma unroll
  for (int t = 0; t < kL1TJ; ++t) {
    if (t < ntj) zhat[((static_cast<size_t>(i) * nj + j0 + t) * two_Q + q) * Hs + zeta] = acc[t];
  }
}

// Step 3: X(s, r) = Re sum_zeta Y'(s, zeta) Z(zeta, r) over a 64 x 64 tile of one pair.
constexpr int kS3Tile = 64;
constexpr int kS3Chunk = 32;  // zeta per shared-memory stage

__device__ __forceinline__ unsigned int float_order_key(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// With `list` the reported template of chunk-local template jl is list[i * nj + jl];
// with `center`, shifts farther than `window` pixels (max norm) from center[i] are skipped.
// The pose index of a key counts templates from `jbase` (key_pos = 0) or by list
// position jl (key_pos = 1), so that one chunk's indices stay below 2^32.
__global__ void __launch_bounds__(256) k_step3_simt(
    const float2* __restrict__ z, const float2* __restrict__ Y, int Hh, int N, int two_Q, int nj, int i0,
    int j0, int NT, float* __restrict__ scores, unsigned long long* __restrict__ keys, const int* __restrict__ list,
    const float2* __restrict__ shifts, const float2* __restrict__ center, float window, int jbase, int key_pos) {
  __shared__ float2 ys[kS3Chunk][kS3Tile];
  __shared__ float2 zs[kS3Chunk][kS3Tile];
  __shared__ unsigned long long red[256];
  const int pair = blockIdx.x;
  const int s0 = blockIdx.y * kS3Tile;
  const int r0 = blockIdx.z * kS3Tile;
  const int tid = threadIdx.x;
  const int ts = tid >> 4, tr = tid & 15;  // 16 x 16 threads, 4 x 4 outputs each
  const float2* zp = z + static_cast<size_t>(pair) * Hh * two_Q;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  for (int c0 = 0; c0 < Hh; c0 += kS3Chunk) {
    const int nc = min(kS3Chunk, Hh - c0);
    for (int e = tid; e < kS3Chunk * kS3Tile; e += 256) {
      const int c = e / kS3Tile, x = e - c * kS3Tile;
      const bool okc = c < nc;
      ys[c][x] = (okc && s0 + x < N) ? Y[static_cast<size_t>(s0 + x) * Hh + c0 + c] : make_float2(0.f, 0.f);
      zs[c][x] = (okc && r0 + x < two_Q) ? zp[static_cast<size_t>(c0 + c) * two_Q + r0 + x] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int c = 0; c < nc; ++c) {
      float2 yv[4], zv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) yv[u] = ys[c][ts * 4 + u];
#pragma unroll
      for (int v = 0; v < 4; ++v) zv[v] = zs[c][tr * 4 + v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(yv[u].x, zv[v].x, fmaf(-yv[u].y, zv[v].y, acc[u][v]));
    }
    __syncthreads();
  }
  const int il = pair / nj, jl = pair - il * nj;
  const int i = i0 + il;
  const int j = list ? __ldg(list + static_cast<size_t>(i) * nj + jl) : j0 + jl;
  if (scores) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = s0 + ts * 4 + u;
      if (s >= N) continue;
      float* row = scores + ((static_cast<size_t>(i) * NT + j) * N + s) * two_Q;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int r = r0 + tr * 4 + v;
        if (r < two_Q) row[r] = acc[u][v];
      }
    }
  }
  if (keys) {
    const unsigned int jk = static_cast<unsigned int>(key_pos ? jl : j - jbase);
    unsigned long long best = 0ull;
    float2 cen = make_float2(0.f, 0.f);
    if (center) cen = center[i];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = s0 + ts * 4 + u;
      bool in_window = s < N;
      if (center && in_window) {
        const float2 sh = shifts[s];
        in_window = fabsf(sh.x - cen.x) <= window && fabsf(sh.y - cen.y) <= window;
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int r = r0 + tr * 4 + v;
        if (in_window && r < two_Q) {
          const unsigned int idx = (jk * two_Q + r) * static_cast<unsigned int>(N) + s;
          const unsigned long long k =
              (static_cast<unsigned long long>(float_order_key(acc[u][v])) << 32) | (0xFFFFFFFFu - idx);
          best = k > best ? k : best;
        }
      }
    }
    red[tid] = best;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (tid < w) red[tid] = red[tid] > red[tid + w] ? red[tid] : red[tid + w];
      __syncthreads();
    }
    if (tid == 0) atomicMax(keys + i, red[0]);
  }
}

// Copies a shortlist, replacing indices outside [0, NT) by 0 and latching kErrIndex.
__global__ void k_sanitize_list(const int* __restrict__ in, long long n, int NT, int* __restrict__ out,
                                int* __restrict__ err) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int j = in[e];
    const bool ok = j >= 0 && j < NT;
    out[e] = ok ? j : 0;
    if (!ok) atomicOr(err, kErrIndex);
  }
}

__global__ void k_best_init(unsigned long long* keys, int NI) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NI) keys[i] = 0ull;
}

// Key = order-preserving score bits (high word) | complemented pose index (low word);
// 0 = no pose scored. Decodes a key into (template offset, rotation, shift, score).
__device__ __forceinline__ void decode_key(unsigned long long k, int N, int two_Q, unsigned int* jr_out,
                                           unsigned int* r_out, unsigned int* s_out, float* score) {
  const unsigned int idx = 0xFFFFFFFFu - static_cast<unsigned int>(k & 0xFFFFFFFFull);
  const unsigned int hi = static_cast<unsigned int>(k >> 32);
  const unsigned int u = (hi & 0x80000000u) ? (hi & 0x7FFFFFFFu) : ~hi;
  const unsigned int jr = idx / static_cast<unsigned int>(N);
  *s_out = idx % static_cast<unsigned int>(N);
  *jr_out = jr / two_Q;
  *r_out = jr % two_Q;
  *score = __uint_as_float(u);
}

// An image whose key is still 0 had no pose scored (every shift outside its window):
// its outputs are template = rotation = shift = -1 and score = -inf, and kErrIndex is
// latched.
__global__ void k_best_finalize(const unsigned long long* __restrict__ keys, int NI, int N, int two_Q,
                                int* tpl, int* rot, int* shift, float* score, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NI) return;
  const unsigned long long k = keys[i];
  if (!k) {
    tpl[i] = rot[i] = shift[i] = -1;
    score[i] = -INFINITY;
    atomicOr(err, kErrIndex);
    return;
  }
  unsigned int j, r, s;
  float v;
  decode_key(k, N, two_Q, &j, &r, &s, &v);
  tpl[i] = static_cast<int>(j);
  rot[i] = static_cast<int>(r);
  shift[i] = static_cast<int>(s);
  score[i] = v;
}

// Pose searches whose pose index can reach 2^32 (NT * R * N) keep per-image records in
// the outputs: set to "none" here, then merged chunk by chunk (k_best_merge).
__global__ void k_best_init_records(unsigned long long* keys, int NI, int* tpl, int* rot, int* shift,
                                    float* score) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NI) return;
  keys[i] = 0ull;
  tpl[i] = rot[i] = shift[i] = -1;
  score[i] = -INFINITY;
}

// Merges the keys of one chunk (images i0 .. i0+ni-1) into the records and clears them.
// The key's template offset is counted from jbase, or is a position in the image's
// list (list != NULL, K entries per image). Chunks come in increasing template order
// (or, for lists, each image's list in one chunk), so a later chunk replaces the record
// only with a strictly larger score: equal scores keep the lower template index, as the
// single-key search does. With `last`, an image left without any pose latches kErrIndex.
__global__ void k_best_merge(unsigned long long* __restrict__ keys, int i0, int ni, int N, int two_Q, int jbase,
                             const int* __restrict__ list, int K, int* tpl, int* rot, int* shift, float* score,
                             int last, int* err) {
  const int il = blockIdx.x * blockDim.x + threadIdx.x;
  if (il >= ni) return;
  const int i = i0 + il;
  const unsigned long long k = keys[i];
  if (k) {
    unsigned int jr, r, s;
    float v;
    decode_key(k, N, two_Q, &jr, &r, &s, &v);
    const float old = score[i];
    if (tpl[i] < 0 || v > old) {
      tpl[i] = list ? list[static_cast<size_t>(i) * K + jr] : jbase + static_cast<int>(jr);
      rot[i] = static_cast<int>(r);
      shift[i] = static_cast<int>(s);
      score[i] = v;
    }
    keys[i] = 0ull;
  }
  if (last && tpl[i] < 0) atomicOr(err, kErrIndex);
}

}  // namespace

cudaError_t launch_step1_simt(const ftk_plan_s* p, const float2* d_a, int ni, const float2* d_b, int nj,
                              float2* d_zhat, cudaStream_t s, const int* d_list_chunk) {
  dim3 grid((p->Hh * p->two_Q + kS1Threads - 1) / kS1Threads, ni, (nj + kS1TJ - 1) / kS1TJ);
  k_step1_simt<<<grid, kS1Threads, 0, s>>>(d_a, d_b, nj, p->d_G, p->d_l, p->Hh, p->M, p->two_Q, d_zhat, d_list_chunk);
  return cudaGetLastError();
}

cudaError_t launch_step1_list_tc(const ftk_plan_s* p, const float2* d_a, int ni, const float2* d_b, int nj,
                                 const int* d_list_chunk, float2* d_zhat, cudaStream_t s) {
  dim3 grid((p->Hh * p->two_Q + kS1Threads - 1) / kS1Threads, ni, (nj + kL1TJ - 1) / kL1TJ);
  const size_t smem = static_cast<size_t>(p->M) * p->Hh * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_step1_list_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_step1_list_tc<<<grid, kS1Threads, smem, s>>>(d_a, d_b, nj, p->d_G, p->d_l, p->Hh, p->M, p->two_Q, d_zhat,
                                                 d_list_chunk);
  return cudaGetLastError();
}

cudaError_t launch_step3_simt(const ftk_plan_s* p, const float2* d_z, int ni, int nj, int i0, int j0, int NT,
                              float* d_scores, unsigned long long* d_keys, cudaStream_t s, const int* d_list,
                              const float2* d_center, float window, int jbase, int key_pos) {
  dim3 grid(ni * nj, (p->N + kS3Tile - 1) / kS3Tile, (p->two_Q + kS3Tile - 1) / kS3Tile);
  k_step3_simt<<<grid, 256, 0, s>>>(d_z, p->d_Y, p->Hh, p->N, p->two_Q, nj, i0, j0, NT, d_scores, d_keys, d_list,
                                    p->d_shifts, d_center, window, jbase, key_pos);
  return cudaGetLastError();
}

cudaError_t launch_sanitize_list(const ftk_plan_s* p, const int* d_in, long long n, int NT, int* d_out,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long g = std::min<long long>((n + 255) / 256, 152LL * 16);
  k_sanitize_list<<<static_cast<unsigned>(g), 256, 0, s>>>(d_in, n, NT, d_out, p->d_err);
  return cudaGetLastError();
}

cudaError_t launch_best_init(unsigned long long* d_keys, int NI, cudaStream_t s) {
  k_best_init<<<(NI + 255) / 256, 256, 0, s>>>(d_keys, NI);
  return cudaGetLastError();
}

cudaError_t launch_best_finalize(const ftk_plan_s* p, const unsigned long long* d_keys, int NI, int* d_tpl,
                                 int* d_rot, int* d_shift, float* d_score, cudaStream_t s) {
  k_best_finalize<<<(NI + 255) / 256, 256, 0, s>>>(d_keys, NI, p->N, p->n_rot, d_tpl, d_rot, d_shift, d_score,
                                                   p->d_err);
  return cudaGetLastError();
}

cudaError_t launch_best_init_records(unsigned long long* d_keys, int NI, int* d_tpl, int* d_rot, int* d_shift,
                                     float* d_score, cudaStream_t s) {
  k_best_init_records<<<(NI + 255) / 256, 256, 0, s>>>(d_keys, NI, d_tpl, d_rot, d_shift, d_score);
  return cudaGetLastError();
}

cudaError_t launch_best_merge(const ftk_plan_s* p, unsigned long long* d_keys, int i0, int ni, int jbase,
                              const int* d_list, int K, const BestRecords& rec, bool last, cudaStream_t s) {
  if (ni <= 0) return cudaSuccess;
  k_best_merge<<<(ni + 255) / 256, 256, 0, s>>>(d_keys, i0, ni, p->N, p->n_rot, jbase, d_list, K, rec.tpl, rec.rot,
                                                rec.shift, rec.score, last ? 1 : 0, p->d_err);
  return cudaGetLastError();
}

}  // namespace ftk
