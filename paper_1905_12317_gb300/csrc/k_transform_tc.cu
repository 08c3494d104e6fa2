// Polar Fourier transform of pixel images on tcgen05 tensor cores.
//
// eq. (Ahattrap) on the polar grid, separably (x first index, y second):
//   T(P, i) = sum_j Ey[j][P] A_ij          (a GEMM: rows P, columns i, K = j)
//   Ahat(P) = dx^2 sum_i Ex[i][P] T(P, i)  (a row-wise weighted sum in the epilogue)
// with P = (m, p), p < Q (real images: the other half is the conjugate).
// MMA rows are 64 columns P of the polar grid, as Re Ey (rows 0..63) and Im Ey
// (rows 64..127); MMA columns are the n pixel rows i of one image; K = the n
// pixel columns j, split into slices of KS. Both operands are split bf16 hi/lo
// (three products, FP32 accumulation in TMEM): Ey^T is packed once per plan on
// the host from its FP64 values, the images per call into scratch owned by the
// plan. The epilogue multiplies each TMEM row by Ex[i][P] and sums over i inside
// the thread that owns the row; the Re and Im halves add their parts into the
// zeroed output.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ftk_internal.h"
#include "tc_engine.h"
#include "tc_ptx.cuh"

namespace ftk {

namespace {

constexpr int kXRows = 128;   // MMA M: 64 polar columns x (Re, Im)
constexpr int kXCols = 64;    // polar columns per tile

__host__ __device__ inline size_t xcanon(int row, int k, int KS) {
  return static_cast<size_t>(row >> 3) * 8 * KS + static_cast<size_t>(k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

int xform_ks(int n) { return n % 64 == 0 ? 64 : (n % 32 == 0 ? 32 : 16); }

// round-to-nearest-even float -> bf16 bits (host)
uint16_t host_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return static_cast<uint16_t>(u >> 16);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}

float host_bf16_to_float(uint16_t b) {
  const uint32_t u = static_cast<uint32_t>(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// images [B][n][n] float -> [b][slice][n rows i][KS] (hi, lo), K = j
__global__ void k_pack_pixels(const float* __restrict__ img, int B, int n, int KS, uint16_t* __restrict__ hi,
                              uint16_t* __restrict__ lo) {
  const int nkg = n / 8;
  const long long total = static_cast<long long>(B) * n * nkg;
  // (row & 7) fastest, then the K chunk, then the row group: coalesced 16-byte stores
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r7 = static_cast<int>(e & 7);
    long long rest = e >> 3;
    const int kg = static_cast<int>(rest % nkg);
    rest /= nkg;
    const int i = static_cast<int>(rest % (n / 8)) * 8 + r7;
    const int b = static_cast<int>(rest / (n / 8));
    const float* src = img + (static_cast<size_t>(b) * n + i) * n + kg * 8;
    uint32_t h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float f0 = src[2 * u], f1 = src[2 * u + 1];
      const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
      const __nv_bfloat16 l0 = __float2bfloat16_rn(f0 - __bfloat162float(h0));
      const __nv_bfloat16 l1 = __float2bfloat16_rn(f1 - __bfloat162float(h1));
      h[u] = static_cast<uint32_t>(__bfloat16_as_ushort(h0)) | (static_cast<uint32_t>(__bfloat16_as_ushort(h1)) << 16);
      l[u] = static_cast<uint32_t>(__bfloat16_as_ushort(l0)) | (static_cast<uint32_t>(__bfloat16_as_ushort(l1)) << 16);
    }
    const int k = kg * 8;
    const size_t off = static_cast<size_t>(b) * n * n + static_cast<size_t>(k / KS) * n * KS + xcanon(i, k % KS, KS);
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

struct XformArgs {
  const uint16_t* ehi;   // Ey^T pack [tile][slice][128][KS]
  const uint16_t* elo;
  const uint16_t* ihi;   // image pack [b][slice][n][KS]
  const uint16_t* ilo;
  const float2* Ex;      // [n][MQ]
  float2* out;           // [B][M][2Q]
  int B, n, KS, n_slices, n_tiles, MQ, Q, ns;
  float dx2;
  int* err;
};

// Warp roles: 0 = bulk-copy producer (and TMEM allocator), 1 = MMA issuer,
// 2..5 = epilogue (one TMEM lane quadrant each). TC = TMEM columns allocated: 512
// (one CTA per SM), or 256 when two accumulators of n columns fit, so that two CTAs
// share an SM and one's epilogue overlaps the other's MMAs.
template <int TC>
__global__ void __launch_bounds__(192, 1) k_polar_tc(const XformArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t e_part = kXRows * a.KS * 2;
  const uint32_t i_part = a.n * a.KS * 2;
  const uint32_t stage_bytes = 2 * (e_part + i_part);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(a.ns) * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = full + a.ns;
  uint64_t* d_full = empty + a.ns;
  uint64_t* d_empty = d_full + 2;
  uint64_t* done_bar = d_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int dcols = (a.n + 31) / 32 * 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.ns; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&d_full[s], 1);
      tc::mbar_init(&d_empty[s], 128);
    }
    tc::mbar_init(done_bar, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc<TC>(tmem_slot);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int n_units = a.B * a.n_tiles;

  if (warp == 0) {
    if (lane == 0) {
      int us = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const int b = u / a.n_tiles, t = u - b * a.n_tiles;
        for (int sl = 0; sl < a.n_slices; ++sl) {
          const int s = us % a.ns;
          if (!(ok = tc::mbar_wait(&empty[s], ((us / a.ns) & 1) ^ 1, abort_flag, a.err))) break;
          tc::mbar_arrive_expect_tx(&full[s], stage_bytes);
          uint8_t* st = smem + static_cast<size_t>(s) * stage_bytes;
          const size_t eoff = (static_cast<size_t>(t) * a.n_slices + sl) * kXRows * a.KS;
          const size_t ioff = static_cast<size_t>(b) * a.n * a.n + static_cast<size_t>(sl) * a.n * a.KS;
          tc::bulk_g2s(st, a.ehi + eoff, e_part, &full[s]);
          tc::bulk_g2s(st + e_part, a.elo + eoff, e_part, &full[s]);
          tc::bulk_g2s(st + 2 * e_part, a.ihi + ioff, i_part, &full[s]);
          tc::bulk_g2s(st + 2 * e_part + i_part, a.ilo + ioff, i_part, &full[s]);
          ++us;
        }
      }
      if (!ok) {
        volatile int never = 0;
        for (int v = us - a.ns; v < us; ++v)
          if (v >= 0) tc::mbar_wait(&full[v % a.ns], (v / a.ns) & 1, &never, a.err, 100000000ull);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(kXRows, a.n);
      const uint32_t sbo = a.KS * 16;
      int us = 0, ud = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++ud) {
        const int sd = ud & 1;
        if (!(ok = tc::mbar_wait(&d_empty[sd], ((ud >> 1) & 1) ^ 1, abort_flag, a.err))) break;
        const uint32_t d_tmem = tmem_base + sd * dcols;
        for (int sl = 0; sl < a.n_slices; ++sl) {
          const int s = us % a.ns;
          if (!(ok = tc::mbar_wait(&full[s], (us / a.ns) & 1, abort_flag, a.err))) break;
          tc::tc_fence_after();
          const uint32_t st = tc::smem_u32(smem + static_cast<size_t>(s) * stage_bytes);
          const uint32_t e_hi = st, e_lo = st + e_part, i_hi = st + 2 * e_part, i_lo = i_hi + i_part;
          for (int kk = 0; kk < a.KS / 16; ++kk) {
            const uint32_t ko = kk * 256;
            const uint64_t deh = tc::smem_desc(e_hi + ko, 128, sbo);
            const uint64_t dih = tc::smem_desc(i_hi + ko, 128, sbo);
            tc::mma_bf16(d_tmem, deh, dih, idesc, (sl > 0 || kk > 0) ? 1u : 0u);
            tc::mma_bf16(d_tmem, deh, tc::smem_desc(i_lo + ko, 128, sbo), idesc, 1u);
            tc::mma_bf16(d_tmem, tc::smem_desc(e_lo + ko, 128, sbo), dih, idesc, 1u);
          }
          tc::mma_commit(&empty[s]);
          ++us;
        }
        if (!ok) break;
        tc::mma_commit(&d_full[sd]);
      }
      tc::mma_commit(done_bar);
      volatile int never = 0;
      tc::mbar_wait(done_bar, 0, &never, a.err, 200000000ull);
    }
  } else {
    const int quad = warp & 3;       // TMEM lanes 32 quad .. 32 quad + 31
    const int row = quad * 32 + lane;
    const int half = row >> 6;       // 0: Re Ey rows, 1: Im Ey rows
    const int c = row & 63;          // polar column within the tile
    const unsigned FULL = 0xFFFFFFFFu;
    int ud = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++ud) {
      const int b = u / a.n_tiles, t = u - b * a.n_tiles;
      const int P = t * kXCols + c;
      const int sd = ud & 1;
      bool w = tc::mbar_wait(&d_full[sd], (ud >> 1) & 1, abort_flag, a.err);
      if (!(ok = __all_sync(FULL, w))) break;
      tc::tc_fence_after();
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quad * 32) << 16) + sd * dcols;
      float sr = 0.f, si = 0.f;  // sum_i Re Ex * T, sum_i Im Ex * T
      for (int c0 = 0; c0 < a.n; c0 += 32) {
        float v[32];
        tc::tmem_ld32(taddr + c0, v);
        if (c0 + 32 >= a.n) {
          tc::tc_fence_before();
          tc::mbar_arrive(&d_empty[sd]);
        }
        if (P < a.MQ) {
#pragma unroll
          for (int x = 0; x < 32; ++x) {
            if (c0 + x < a.n) {
              const float2 ex = __ldg(a.Ex + static_cast<size_t>(c0 + x) * a.MQ + P);
              sr = fmaf(ex.x, v[x], sr);
              si = fmaf(ex.y, v[x], si);
            }
          }
        }
      }
      // Ahat = sum_i (Ex_r + i Ex_i)(T_r + i T_i): Re = sr(T_r) - si(T_i), Im = si(T_r) + sr(T_i).
      // The Re and Im halves live in different warps; each adds its part to the zeroed
      // output (two addends per value, so the sum does not depend on their order).
      if (P < a.MQ) {
        const int m = P / a.Q, p = P - m * a.Q;
        float2* o = a.out + (static_cast<size_t>(b) * (a.MQ / a.Q) + m) * (2 * a.Q);
        const float dr = a.dx2 * (half ? -si : sr), di = a.dx2 * (half ? sr : si);
        atomicAdd(&o[p].x, dr);
        atomicAdd(&o[p].y, di);
        atomicAdd(&o[p + a.Q].x, dr);
        atomicAdd(&o[p + a.Q].y, -di);
      }
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc<TC>(tmem_base);
}

size_t xform_stage_bytes(int n, int KS) { return 2 * (static_cast<size_t>(kXRows) * KS * 2 + static_cast<size_t>(n) * KS * 2); }

}  // namespace

bool xform_tc_supported(const ftk_plan_s* p) {
  const int n = p->n;
  if (n % 16 != 0 || n > 256 || n < 16) return false;
  return 2 * xform_stage_bytes(n, xform_ks(n)) + 1024 <= 227 * 1024;
}

cudaError_t xform_build_tables(ftk_plan_s* p, const std::vector<double>& ey_re, const std::vector<double>& ey_im) {
  const int n = p->n, MQ = p->M * p->Q, KS = xform_ks(n);
  const int n_tiles = (MQ + kXCols - 1) / kXCols;
  const int n_slices = n / KS;
  std::vector<uint16_t> hi(static_cast<size_t>(n_tiles) * n_slices * kXRows * KS, 0);
  std::vector<uint16_t> lo(hi.size(), 0);
  for (int t = 0; t < n_tiles; ++t)
    for (int r = 0; r < kXRows; ++r) {
      const int P = t * kXCols + (r & 63);
      if (P >= MQ) continue;
      for (int j = 0; j < n; ++j) {
        const double v = (r < 64 ? ey_re : ey_im)[static_cast<size_t>(j) * MQ + P];
        const uint16_t h = host_bf16(static_cast<float>(v));
        const uint16_t l = host_bf16(static_cast<float>(v - static_cast<double>(host_bf16_to_float(h))));
        const size_t off = (static_cast<size_t>(t) * n_slices + j / KS) * kXRows * KS + xcanon(r, j % KS, KS);
        hi[off] = h;
        lo[off] = l;
      }
    }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p->xf.d_ehi), hi.size() * 2);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->xf.d_elo), lo.size() * 2);
  if (e == cudaSuccess) e = cudaMemcpy(p->xf.d_ehi, hi.data(), hi.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->xf.d_elo, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice);
  return e;
}

void xform_free_tables(ftk_plan_s* p) {
  cudaFree(p->xf.d_ehi);
  cudaFree(p->xf.d_elo);
  cudaFree(p->xf.d_pix);
  p->xf.d_ehi = p->xf.d_elo = nullptr;
  p->xf.d_pix = nullptr;
  p->xf.pix_images = 0;
}

// Pixel-pack scratch of the plan: images per transform launch (about 64 MiB of bf16 hi/lo).
int xform_pix_images(int n) { return std::max(1, static_cast<int>((64ll << 20) / (4ll * n * n))); }

cudaError_t xform_alloc_scratch(ftk_plan_s* p) {
  p->xf.pix_images = xform_pix_images(p->n);
  return cudaMalloc(reinterpret_cast<void**>(&p->xf.d_pix), static_cast<size_t>(p->xf.pix_images) * p->n * p->n * 4);
}

ftk_status xform_run(ftk_plan_s* p, const float* d_images, int B, float2* d_out, cudaStream_t s) {
  const int n = p->n, MQ = p->M * p->Q, KS = xform_ks(n);
  const int n_tiles = (MQ + kXCols - 1) / kXCols;
  const int chunk = p->xf.pix_images;
  if (!p->xf.d_pix || chunk < 1) return FTK_ERR_UNSUPPORTED;
  uint16_t* ihi = p->xf.d_pix;
  uint16_t* ilo = ihi + static_cast<size_t>(p->xf.pix_images) * n * n;
  XformArgs args;
  args.ehi = p->xf.d_ehi;
  args.elo = p->xf.d_elo;
  args.ihi = ihi;
  args.ilo = ilo;
  args.Ex = p->d_Ex;
  args.n = n;
  args.KS = KS;
  args.n_slices = n / KS;
  args.n_tiles = n_tiles;
  args.MQ = MQ;
  args.Q = p->Q;
  args.dx2 = static_cast<float>(p->dx * p->dx);
  args.err = p->d_err;
  const size_t stage = xform_stage_bytes(n, KS);
  // two CTAs per SM when two stages of both and two n-column accumulators each fit
  const bool two = 2 * ((n + 31) / 32 * 32) <= 256 && 2 * (2 * stage + 1024) <= 226 * 1024;
  int ns = two ? 2 : 4;
  while (ns > 2 && ns * stage + 1024 > 227 * 1024) --ns;
  args.ns = ns;
  // one CTA per SM: at least half of the shared memory, so that no other CTA shares
  // the SM's 512 TMEM columns; two CTAs: each allocates 256 columns
  const size_t smem = two ? ns * stage + 1024 : std::max<size_t>(ns * stage + 1024, 116 * 1024);
  cudaError_t e = two ? cudaFuncSetAttribute(k_polar_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                      : cudaFuncSetAttribute(k_polar_tc<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return FTK_ERR_CUDA;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  for (int b0 = 0; b0 < B; b0 += chunk) {
    const int nb = std::min(chunk, B - b0);
    const long long total = static_cast<long long>(nb) * n * (n / 8);
    const int g = static_cast<int>(std::min<long long>((total + 255) / 256, 152LL * 32));
    FTK_LAUNCH(p, kKPackPixels, s,
               (k_pack_pixels<<<g, 256, 0, s>>>(d_images + static_cast<size_t>(b0) * n * n, nb, n, KS, ihi, ilo),
                cudaGetLastError()));
    args.B = nb;
    args.out = d_out + static_cast<size_t>(b0) * p->M * 2 * p->Q;
    if (cudaMemsetAsync(args.out, 0, static_cast<size_t>(nb) * p->M * 2 * p->Q * sizeof(float2), s) != cudaSuccess)
      return FTK_ERR_CUDA;
    const int grid = std::min(nb * n_tiles, two ? 2 * nsm : nsm);
    if (two)
      FTK_LAUNCH(p, kKPolarTc, s, (k_polar_tc<256><<<grid, 192, smem, s>>>(args), cudaGetLastError()));
    else
      FTK_LAUNCH(p, kKPolarTc, s, (k_polar_tc<512><<<grid, 192, smem, s>>>(args), cudaGetLastError()));
  }
  return FTK_OK;
}

}  // namespace ftk
