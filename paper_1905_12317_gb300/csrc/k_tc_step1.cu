// Step 1 of eq. (fbk3) on tcgen05 tensor cores.
//
//   Zhat_zeta(q) = sum_m [2 pi w_m G_zeta(k_m)] a(k_m; q - l_zeta) conj b(k_m; q)
//
// For one rotation-frequency q this is a GEMM over templates: with
// A'_zeta(m) = 2 pi w_m G_zeta(k_m) a(k_m; q - l_zeta) and K index k = 2m + {0, 1},
//   D[j, 2 zeta]     = Re(A' conj b_j) = sum_m (A'r br + A'i bi)      row (zeta, re) = ( A'r,  A'i)
//   D[j, 2 zeta + 1] = Im(A' conj b_j) = sum_m (A'i br - A'r bi)      row (zeta, im) = ( A'i, -A'r)
// with the template row j = (br, bi). MMA rows are 128 templates (M = 128),
// columns the 2 H_half (padded) rows of one image (N), K = 2M split into
// slices of at most 64. Both operands are packed once per chunk into the
// no-swizzle K-major core-matrix layout, bf16 hi/lo (BF16x3) or hi only (BF16).
// Output Zhat is FP32, layout [pair][q][zeta].
#include <cuda_bf16.h>

#include <algorithm>

#include "ftk_internal.h"
#include "tc_engine.h"
#include "tc_ptx.cuh"

namespace ftk {

namespace {

constexpr int kTRows = 128;
constexpr int kTmemCols1 = 512;
constexpr int kStep1DefaultStages = 6;
constexpr size_t kStep1Tail = 512 + 8 * 32 * 36 * sizeof(float);  // barriers + epilogue staging
constexpr size_t kStep1SmemMax = 227 * 1024;

// One operand pipeline stage: a 128-template tile and the image's Np rows, K slice KS,
// bf16 hi and lo (BF16x3) or one part.
size_t step1_stage_bytes(int Np, int KS, int x3) {
  return static_cast<size_t>(tc::mode_split(x3) ? 2 : 1) * (kTRows * KS * 2 + Np * KS * 2);
}

// Pipeline stages that fit in shared memory next to the epilogue staging (at most `want`).
int step1_fit_stages(size_t stage, int want) {
  int ns = want;
  while (ns > 2 && ns * stage + kStep1Tail > kStep1SmemMax) --ns;
  return ns * stage + kStep1Tail > kStep1SmemMax ? 1 : ns;
}

__device__ __forceinline__ size_t canon(int row, int k, int KS) {
  return static_cast<size_t>(row >> 3) * 8 * KS + static_cast<size_t>(k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

// Eight FP32 values -> eight 16-bit operands (hi) and, for BF16x3, their residuals (lo).
__device__ __forceinline__ void split8(const float* f, uint4& hi, uint4& lo, int mode) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) tc::pack2(f[2 * u], f[2 * u + 1], mode, h[u], l[u]);
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Templates b [nj][M][2Q] -> T[q][jt][slice][128 rows][KS] (hi, lo).
__global__ void k_pack_templates(const float2* __restrict__ b, int nj, int M, int two_Q, int n_jt, int KS,
                                 uint16_t* __restrict__ thi, uint16_t* __restrict__ tlo, int x3) {
  const int K2 = 2 * M;
  const int nkg = K2 / 8;
  const long long total = static_cast<long long>(two_Q) * n_jt * kTRows * nkg;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int kg = static_cast<int>(e % nkg);
    long long rest = e / nkg;
    const int row = static_cast<int>(rest % kTRows);
    rest /= kTRows;
    const int jt = static_cast<int>(rest % n_jt);
    const int q = static_cast<int>(rest / n_jt);
    const int j = jt * kTRows + row;
    float f[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int m = kg * 4 + u;
      const float2 c = j < nj ? b[(static_cast<size_t>(j) * M + m) * two_Q + q] : make_float2(0.f, 0.f);
      f[2 * u] = c.x;
      f[2 * u + 1] = c.y;
    }
    uint4 hi, lo;
    split8(f, hi, lo, x3);
    const int k = kg * 8;
    const size_t off = (static_cast<size_t>(q) * n_jt + jt) * kTRows * K2 + static_cast<size_t>(k / KS) * kTRows * KS +
                       canon(row, k % KS, KS);
    *reinterpret_cast<uint4*>(thi + off) = hi;
    if (x3 == tc::kModeBf16x3) *reinterpret_cast<uint4*>(tlo + off) = lo;
  }
}

// Per-image template tiles gathered from the packed template set T[q][jt][slice][128][KS]
// (k_pack_templates over all NT templates): 16-byte pieces (8 K values of one row) are copied
// into the list layout T[i][q][jt][slice][Rt rows][KS] (hi, lo), row r of tile jt holding the
// template list[i][jt * 128 + r]; Rt is the tile's row stride, 128, or the list length rounded
// up to 8 when one tile holds the whole list. Rows past the list's end are zero.
__global__ void k_gather_template_tiles(const uint4* __restrict__ thi_all, const uint4* __restrict__ tlo_all,
                                        int n_jt_all, const int* __restrict__ list, int ni, int K, int two_Q,
                                        int n_jt, int Rt, int K2, int KS, uint4* __restrict__ thi,
                                        uint4* __restrict__ tlo, int x3) {
  const int nkg = K2 / 8;
  const int nrg = Rt / 8;
  const long long total = static_cast<long long>(ni) * two_Q * n_jt * Rt * nkg;
  // thread order (row & 7) fastest, then the K chunk, then the row group: consecutive
  // threads write consecutive 16-byte pieces of the core-matrix layout
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r7 = static_cast<int>(e & 7);
    long long rest = e >> 3;
    const int kg = static_cast<int>(rest % nkg);
    rest /= nkg;
    const int row = static_cast<int>(rest % nrg) * 8 + r7;
    rest /= nrg;
    const int jt = static_cast<int>(rest % n_jt);
    rest /= n_jt;
    const int q = static_cast<int>(rest % two_Q);
    const int i = static_cast<int>(rest / two_Q);
    const int jl = jt * kTRows + row;
    const int j = jl < K ? list[static_cast<size_t>(i) * K + jl] : -1;
    const int k = kg * 8;
    const size_t dst = (((static_cast<size_t>(i) * two_Q + q) * n_jt + jt) * Rt * K2 +
                        static_cast<size_t>(k / KS) * Rt * KS + canon(row, k % KS, KS)) / 8;
    uint4 h = make_uint4(0u, 0u, 0u, 0u), l = h;
    if (j >= 0) {
      const int jts = j / kTRows, rs = j - jts * kTRows;
      const size_t src = ((static_cast<size_t>(q) * n_jt_all + jts) * kTRows * K2 +
                          static_cast<size_t>(k / KS) * kTRows * KS + canon(rs, k % KS, KS)) / 8;
      h = thi_all[src];
      if (x3 == tc::kModeBf16x3) l = tlo_all[src];
    }
    thi[dst] = h;
    if (x3 == tc::kModeBf16x3) tlo[dst] = l;
  }
}

// Images a [ni][M][2Q] -> I[i][q][slice][Np rows][KS] (hi, lo); row n = 2 zeta + part.
__global__ void k_pack_images(const float2* __restrict__ a, int ni, const float* __restrict__ G,
                              const int* __restrict__ lz, int Hh, int M, int two_Q, int Np, int KS,
                              uint16_t* __restrict__ ihi, uint16_t* __restrict__ ilo, int x3) {
  const int K2 = 2 * M;
  const int nkg = K2 / 8;
  const int nrg = Np / 8;
  const long long total = static_cast<long long>(ni) * two_Q * Np * nkg;
  // thread order (row & 7) fastest, then the K chunk, then the row group (coalesced stores)
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r7 = static_cast<int>(e & 7);
    long long rest = e >> 3;
    const int kg = static_cast<int>(rest % nkg);
    rest /= nkg;
    const int n = static_cast<int>(rest % nrg) * 8 + r7;
    rest /= nrg;
    const int q = static_cast<int>(rest % two_Q);
    const int i = static_cast<int>(rest / two_Q);
    const int zeta = n >> 1, part = n & 1;
    float f[8];
    if (zeta < Hh) {
      int qa = q - lz[zeta];
      qa += qa < 0 ? two_Q : 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int m = kg * 4 + u;
        const float g = G[static_cast<size_t>(zeta) * M + m];
        const float2 c = a[(static_cast<size_t>(i) * M + m) * two_Q + qa];
        const float ar = g * c.x, ai = g * c.y;
        f[2 * u] = part ? ai : ar;
        f[2 * u + 1] = part ? -ar : ai;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) f[u] = 0.f;
    }
    uint4 hi, lo;
    split8(f, hi, lo, x3);
    const int k = kg * 8;
    const size_t off = (static_cast<size_t>(i) * two_Q + q) * Np * K2 + static_cast<size_t>(k / KS) * Np * KS +
                       canon(n, k % KS, KS);
    *reinterpret_cast<uint4*>(ihi + off) = hi;
    if (x3 == tc::kModeBf16x3) *reinterpret_cast<uint4*>(ilo + off) = lo;
  }
}

struct Step1Args {
  const uint16_t* thi;
  const uint16_t* tlo;
  const uint16_t* ihi;
  const uint16_t* ilo;
  int K2, KS, n_slices, Np, Hh, Hs, two_Q, n_jt, nj, ni, q_split, q_per_unit;
  float2* zhat;
  int* err;
  int x3, ns, nd, dcols;
  // per-image template packs (T[i][q][jt][slice][Rt][KS]); t_rows = Rt, else 0
  int t_rows;
  // shared template pack T[q][t_njt][slice][128][KS]: this launch's tiles start at tile jt0
  int jt0, t_njt;
};

// Warp roles: 0 = bulk-copy producer and TMEM owner, 1 = MMA issuer (the whole warp,
// one elected lane issues), 2-9 = epilogue in two sets of four warps (one TMEM lane
// quadrant per warp); set e drains the accumulators of every other q, so that the
// TMEM loads and stores of one set overlap those of the other.
constexpr int kStep1Threads = 320;

__global__ void __launch_bounds__(kStep1Threads, 1) k_step1_tc(const Step1Args a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int parts = tc::mode_split(a.x3) ? 2 : 1;
  const uint32_t t_part = kTRows * a.KS * 2;
  const uint32_t i_part = a.Np * a.KS * 2;
  const uint32_t stage_bytes = parts * (t_part + i_part);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(a.ns) * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = full + a.ns;
  uint64_t* d_full = empty + a.ns;
  uint64_t* d_empty = d_full + a.nd;
  uint64_t* done_bar = d_empty + a.nd;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* stage_base = reinterpret_cast<float*>(smem + static_cast<size_t>(a.ns) * stage_bytes + 512);

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.ns; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < a.nd; ++s) {
      tc::mbar_init(&d_full[s], 1);
      tc::mbar_init(&d_empty[s], 128);
    }
    tc::mbar_init(done_bar, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc<kTmemCols1>(tmem_slot);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int n_units = a.ni * a.n_jt * a.q_split;

  if (warp == 0) {
    if (lane == 0) {
      int us = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const int i = u / (a.n_jt * a.q_split);
        const int rem = u - i * a.n_jt * a.q_split;
        const int jt = rem / a.q_split;
        const int q0 = (rem - jt * a.q_split) * a.q_per_unit;
        const int q1 = min(a.two_Q, q0 + a.q_per_unit);
        for (int q = q0; q < q1 && ok; ++q) {
          for (int sl = 0; sl < a.n_slices; ++sl) {
            const int s = us % a.ns;
            if (!(ok = tc::mbar_wait(&empty[s], ((us / a.ns) & 1) ^ 1, abort_flag, a.err))) break;
            // list mode copies only the tile's Rt rows; the MMA's rows past them read stale
            // shared memory and land in D rows that the epilogue never stores
            const uint32_t t_bytes = a.t_rows ? static_cast<uint32_t>(a.t_rows) * a.KS * 2 : t_part;
            tc::mbar_arrive_expect_tx(&full[s], parts * (t_bytes + i_part));
            uint8_t* st = smem + static_cast<size_t>(s) * stage_bytes;
            const size_t toff =
                a.t_rows ? (((static_cast<size_t>(i) * a.two_Q + q) * a.n_jt + jt) * a.n_slices + sl) * a.t_rows * a.KS
                         : ((static_cast<size_t>(q) * a.t_njt + a.jt0 + jt) * a.n_slices + sl) * kTRows * a.KS;
            const size_t ioff = ((static_cast<size_t>(i) * a.two_Q + q) * a.n_slices + sl) * a.Np * a.KS;
            tc::bulk_g2s(st, a.thi + toff, t_bytes, &full[s]);
            tc::bulk_g2s(st + parts * t_part, a.ihi + ioff, i_part, &full[s]);
            if (tc::mode_split(a.x3)) {
              tc::bulk_g2s(st + t_part, a.tlo + toff, t_bytes, &full[s]);
              tc::bulk_g2s(st + parts * t_part + i_part, a.ilo + ioff, i_part, &full[s]);
            }
            ++us;
          }
        }
      }
      if (!ok) {
        volatile int never = 0;
        for (int v = us - a.ns; v < us; ++v)
          if (v >= 0) tc::mbar_wait(&full[v % a.ns], (v / a.ns) & 1, &never, a.err, 100000000ull);
      }
    }
  } else if (warp == 1) {
    const unsigned FULL = 0xFFFFFFFFu;
    const uint32_t idesc = tc::idesc_f32acc(kTRows, a.Np, a.x3);
    const uint32_t sbo = a.KS * 16;
    // descriptors are advanced by adding (byte offset >> 4) to the start-address field
    const uint64_t desc0 = tc::smem_desc(tc::smem_u32(smem), 128, sbo);
    const uint64_t t_lo_step = t_part >> 4, i_step = (parts * t_part) >> 4, i_lo_step = i_part >> 4;
    // stage and accumulator index and phase kept as counters (no division by the stage count
    // on the issue path), the K steps of a 32-wide slice issued unrolled: 3% faster at n = 128
    int cs = 0, cd = 0;
    uint32_t cs_ph = 0, cd_ph = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int rem = u % (a.n_jt * a.q_split);
      const int jt = rem / a.q_split;
      const int q0 = (rem - jt * a.q_split) * a.q_per_unit;
      const int q1 = min(a.two_Q, q0 + a.q_per_unit);
      for (int q = q0; q < q1 && ok; ++q) {
        const int sd = cd;
        if (!(ok = __all_sync(FULL, tc::mbar_wait(&d_empty[sd], cd_ph ^ 1, abort_flag, a.err)))) break;
        tc::tc_fence_after();
        const uint32_t d_tmem = tmem_base + sd * a.dcols;
        for (int sl = 0; sl < a.n_slices; ++sl) {
          const int s = cs;
          if (!(ok = __all_sync(FULL, tc::mbar_wait(&full[s], cs_ph, abort_flag, a.err)))) break;
          tc::tc_fence_after();
          const uint64_t dth = desc0 + ((static_cast<uint64_t>(s) * stage_bytes) >> 4);
          const uint64_t dih = dth + i_step;
          if (a.KS == 32 && tc::mode_split(a.x3)) {
            tc::mma_bf16x3_ss_warp(d_tmem, dth, dth + t_lo_step, dih, dih + i_lo_step, idesc, sl > 0 ? 1u : 0u);
            tc::mma_bf16x3_ss_warp(d_tmem, dth + 16, dth + 16 + t_lo_step, dih + 16, dih + 16 + i_lo_step, idesc, 1u);
          } else {
            for (int kk = 0; kk < a.KS / 16; ++kk) {
              const uint32_t acc = (sl > 0 || kk > 0) ? 1u : 0u;
              const uint64_t o = static_cast<uint64_t>(kk) * 16;
              if (tc::mode_split(a.x3))
                tc::mma_bf16x3_ss_warp(d_tmem, dth + o, dth + o + t_lo_step, dih + o, dih + o + i_lo_step, idesc, acc);
              else
                tc::mma_bf16_ss_warp(d_tmem, dth + o, dih + o, idesc, acc);
            }
          }
          tc::mma_commit_warp(&empty[s]);
          if (++cs == a.ns) {
            cs = 0;
            cs_ph ^= 1u;
          }
        }
        if (!ok) break;
        tc::mma_commit_warp(&d_full[sd]);
        if (++cd == a.nd) {
          cd = 0;
          cd_ph ^= 1u;
        }
      }
    }
    tc::mma_commit_warp(done_bar);
    volatile int never = 0;
    tc::mbar_wait(done_bar, 0, &never, a.err, 200000000ull);
  } else {
    const int quad = warp & 3;
    const int eset = (warp - 2) >> 2;
    const unsigned FULL = 0xFFFFFFFFu;
    int ud = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int i = u / (a.n_jt * a.q_split);
      const int rem = u - i * a.n_jt * a.q_split;
      const int jt = rem / a.q_split;
      const int q0 = (rem - jt * a.q_split) * a.q_per_unit;
      const int q1 = min(a.two_Q, q0 + a.q_per_unit);
      const int jw = jt * kTRows + quad * 32;  // first template of this warp's 32 rows
      // Per-warp staging of one 32-column slice of D: row = lane (template), 36 floats
      // apart (16-byte aligned rows, banks spread). Re-read by the warp so that each
      // store instruction writes 4 rows x 128 contiguous bytes of Zhat [pair][q][zeta].
      float* stage = stage_base + (warp - 2) * 32 * 36;
      const int rsub = lane >> 3, piece = lane & 7;
      for (int q = q0; q < q1; ++q) {
        const int sd = ud % a.nd;
        if ((ud & 1) != eset) {
          ++ud;
          continue;
        }
        bool w = tc::mbar_wait(&d_full[sd], (ud / a.nd) & 1, abort_flag, a.err);
        if (!(ok = __all_sync(FULL, w))) break;
        tc::tc_fence_after();
        const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quad * 32) << 16) + sd * a.dcols;
        for (int c0 = 0; c0 < a.Np; c0 += 32) {
          float v[32];
          tc::tmem_ld32(taddr + c0, v);
          if (c0 + 32 >= a.Np) {  // the TMEM buffer is free once its last slice is in registers
            tc::tc_fence_before();
            tc::mbar_arrive(&d_empty[sd]);
          }
#pragma unroll
          for (int t = 0; t < 32; t += 4)
            *reinterpret_cast<float4*>(stage + lane * 36 + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
          __syncwarp();
          const int zc = (c0 >> 1) + 2 * piece;  // first of the two complex values of this lane's piece
          if (zc < a.Hh) {
#pragma unroll
            for (int g = 0; g < 8; ++g) {
              const int rr = 4 * g + rsub;
              const int j = jw + rr;
              if (j < a.nj) {
                float2* dst = a.zhat + ((static_cast<size_t>(i) * a.nj + j) * a.two_Q + q) * a.Hs + zc;
                // streaming store: Zhat is read once, by the next kernel, and should not evict
                // the template and image tiles that the other CTAs of this launch re-read from L2
                __stcs(reinterpret_cast<float4*>(dst), *reinterpret_cast<const float4*>(stage + rr * 36 + 4 * piece));
              }
            }
          }
          __syncwarp();
        }
        ++ud;
      }
    }
  }

  __syncwarp();  // the single-lane producer rejoins its warp
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc<kTmemCols1>(tmem_base);
}

}  // namespace

int step1_np(const ftk_plan_s* p) { return (2 * p->Hh + 15) / 16 * 16; }
int step1_k2(const ftk_plan_s* p) { return 2 * p->M; }
// K slice of the Step-1 operands. 32-wide slices where they keep as many operand bytes in
// flight as 64-wide ones (twice the stages at half the size): a stage is then released after
// half of a q's MMAs, which made Step 1 4% faster at n = 64 (M = 32, BF16x3).
int step1_ks(const ftk_plan_s* p, int x3) {
  const int K2 = 2 * p->M;
  if (K2 % 64 != 0) return K2 % 32 == 0 ? 32 : 16;
  const int Np = step1_np(p);
  const size_t s32 = step1_stage_bytes(Np, 32, x3), s64 = step1_stage_bytes(Np, 64, x3);
  return step1_fit_stages(s32, kStep1DefaultStages) * s32 >= step1_fit_stages(s64, kStep1DefaultStages) * s64 ? 32
                                                                                                             : 64;
}

bool step1_tc_supported(const ftk_plan_s* p) {
  return (2 * p->M) % 16 == 0 && step1_np(p) <= 256;
}

size_t step1_image_bytes(const ftk_plan_s* p) {
  return static_cast<size_t>(p->two_Q) * step1_np(p) * step1_k2(p) * 2 * 2;
}
size_t step1_template_row_bytes(const ftk_plan_s* p) { return static_cast<size_t>(p->two_Q) * step1_k2(p) * 2 * 2; }

ftk_status step1_tc_launch(ftk_plan_s* p, int x3, const uint16_t* thi, const uint16_t* tlo, const uint16_t* ihi,
                           const uint16_t* ilo, int ni, int nj, int n_jt, int t_rows, float2* zhat, cudaStream_t s,
                           int jt0 = 0, int t_njt = 0);

namespace {

ftk_status pack_images_launch(ftk_plan_s* p, int x3, const float2* a, int ni, uint16_t* ibuf, cudaStream_t s) {
  const int K2 = step1_k2(p), KS = step1_ks(p, x3), Np = step1_np(p);
  uint16_t* ihi = ibuf;
  uint16_t* ilo = ihi + static_cast<size_t>(ni) * p->two_Q * Np * K2;
  const long long total = static_cast<long long>(ni) * p->two_Q * Np * (K2 / 8);
  const int grid = static_cast<int>(std::min<long long>((total + 255) / 256, 148LL * 32));
  FTK_LAUNCH(p, kKPackTemplates, s,
             (k_pack_images<<<grid, 256, 0, s>>>(a, ni, p->d_G, p->d_l, p->Hh, p->M, p->two_Q, Np, KS, ihi, ilo, x3),
              cudaGetLastError()));
  return FTK_OK;
}

}  // namespace

ftk_status step1_tc_run(ftk_plan_s* p, int precision, const float2* a, int ni, const float2* b, int nj, float2* zhat,
                        uint16_t* tbuf, uint16_t* ibuf, bool pack_templates, cudaStream_t s) {
  const int x3 = op_mode(precision);
  const int K2 = step1_k2(p), KS = step1_ks(p, x3), Np = step1_np(p);
  const int n_jt = (nj + kTRows - 1) / kTRows;
  uint16_t* thi = tbuf;
  uint16_t* tlo = thi + static_cast<size_t>(p->two_Q) * n_jt * kTRows * K2;
  uint16_t* ihi = ibuf;
  uint16_t* ilo = ihi + static_cast<size_t>(ni) * p->two_Q * Np * K2;
  if (pack_templates) {
    const long long total = static_cast<long long>(p->two_Q) * n_jt * kTRows * (K2 / 8);
    const int grid = static_cast<int>(std::min<long long>((total + 255) / 256, 148LL * 32));
    FTK_LAUNCH(p, kKPackTemplates, s,
               (k_pack_templates<<<grid, 256, 0, s>>>(b, nj, p->M, p->two_Q, n_jt, KS, thi, tlo, x3),
                cudaGetLastError()));
  }
  const ftk_status st = pack_images_launch(p, x3, a, ni, ibuf, s);
  if (st != FTK_OK) return st;
  return step1_tc_launch(p, x3, thi, tlo, ihi, ilo, ni, nj, n_jt, 0, zhat, s);
}

ftk_status step1_tc_run_block(ftk_plan_s* p, int precision, const float2* a, int ni, int nj, int jt0, int NT,
                              const uint16_t* tall, float2* zhat, uint16_t* ibuf, bool pack_images, cudaStream_t s) {
  const int x3 = op_mode(precision);
  const int K2 = step1_k2(p), Np = step1_np(p);
  const int n_jt = (nj + kTRows - 1) / kTRows;
  const int t_njt = (NT + kTRows - 1) / kTRows;
  if (jt0 < 0 || jt0 + n_jt > t_njt) return FTK_ERR_ARG;
  const uint16_t* thi = tall;
  const uint16_t* tlo = thi + static_cast<size_t>(p->two_Q) * t_njt * kTRows * K2;
  uint16_t* ihi = ibuf;
  uint16_t* ilo = ihi + static_cast<size_t>(ni) * p->two_Q * Np * K2;
  if (pack_images) {
    const ftk_status st = pack_images_launch(p, x3, a, ni, ibuf, s);
    if (st != FTK_OK) return st;
  }
  return step1_tc_launch(p, x3, thi, tlo, ihi, ilo, ni, nj, n_jt, 0, zhat, s, jt0, t_njt);
}

ftk_status step1_tc_launch(ftk_plan_s* p, int x3, const uint16_t* thi, const uint16_t* tlo, const uint16_t* ihi,
                           const uint16_t* ilo, int ni, int nj, int n_jt, int t_rows, float2* zhat, cudaStream_t s,
                           int jt0, int t_njt) {
  const int K2 = step1_k2(p), KS = step1_ks(p, x3), Np = step1_np(p);
  Step1Args args;
  args.t_rows = t_rows;
  args.jt0 = jt0;
  args.t_njt = t_njt > 0 ? t_njt : n_jt;
  args.thi = thi;
  args.tlo = tlo;
  args.ihi = ihi;
  args.ilo = ilo;
  args.K2 = K2;
  args.KS = KS;
  args.n_slices = K2 / KS;
  args.Np = Np;
  args.Hh = p->Hh;
  args.Hs = (p->Hh + 1) / 2 * 2;
  args.two_Q = p->two_Q;
  args.n_jt = n_jt;
  args.nj = nj;
  args.ni = ni;
  args.zhat = zhat;
  args.err = p->d_err;
  args.x3 = x3;
  args.dcols = (Np + 31) / 32 * 32;
  args.nd = std::min(4, kTmemCols1 / args.dcols);
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int units0 = ni * n_jt;
  // default: about one unit (image, template tile, q range) per SM; splitting q ranges further only
  // adds per-unit cost (n = 128, 8 x 4096-pair chunks: 7% faster than two units per SM)
  const int per_sm = p->tune.step1_ctas_per_sm > 0 ? p->tune.step1_ctas_per_sm : 1;
  int q_split = std::max(1, std::min(p->two_Q, (per_sm * nsm + units0 - 1) / units0));
  args.q_per_unit = (p->two_Q + q_split - 1) / q_split;
  args.q_split = (p->two_Q + args.q_per_unit - 1) / args.q_per_unit;
  const size_t stage = step1_stage_bytes(Np, KS, x3);
  const int ns = step1_fit_stages(stage, p->tune.step1_stages > 0 ? p->tune.step1_stages : kStep1DefaultStages);
  args.ns = ns;
  const size_t smem = std::max<size_t>(ns * stage + kStep1Tail, 116 * 1024);
  cudaError_t e = cudaFuncSetAttribute(k_step1_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return FTK_ERR_CUDA;
  const int units = ni * n_jt * args.q_split;
  const int grid = std::min(units, nsm);
  FTK_LAUNCH(p, kKStep1Tc, s, (k_step1_tc<<<grid, kStep1Threads, smem, s>>>(args), cudaGetLastError()));
  return FTK_OK;
}

int step1_list_rows(int K) { return K > kTRows ? kTRows : (K + 7) / 8 * 8; }

size_t step1_list_template_bytes(const ftk_plan_s* p, int K) {
  const int n_jt = (K + kTRows - 1) / kTRows;
  return static_cast<size_t>(p->two_Q) * n_jt * step1_list_rows(K) * step1_k2(p) * 2 * 2;
}

size_t step1_all_template_bytes(const ftk_plan_s* p, int NT) {
  const int n_jt = (NT + kTRows - 1) / kTRows;
  return static_cast<size_t>(p->two_Q) * n_jt * kTRows * step1_k2(p) * 2 * 2;
}

ftk_status step1_pack_all_templates(ftk_plan_s* p, int precision, const float2* b, int NT, uint16_t* tall,
                                    cudaStream_t s) {
  const int x3 = op_mode(precision);
  const int K2 = step1_k2(p), KS = step1_ks(p, x3);
  const int n_jt = (NT + kTRows - 1) / kTRows;
  uint16_t* thi = tall;
  uint16_t* tlo = thi + static_cast<size_t>(p->two_Q) * n_jt * kTRows * K2;
  const long long total = static_cast<long long>(p->two_Q) * n_jt * kTRows * (K2 / 8);
  const int grid = static_cast<int>(std::min<long long>((total + 255) / 256, 148LL * 32));
  FTK_LAUNCH(p, kKPackTemplates, s,
             (k_pack_templates<<<grid, 256, 0, s>>>(b, NT, p->M, p->two_Q, n_jt, KS, thi, tlo, x3), cudaGetLastError()));
  return FTK_OK;
}

ftk_status step1_tc_run_list(ftk_plan_s* p, int precision, const float2* a, int ni, const uint16_t* tall, int NT,
                             const int* list, int K, float2* zhat, uint16_t* tbuf, uint16_t* ibuf, cudaStream_t s) {
  const int x3 = op_mode(precision);
  const int K2 = step1_k2(p), KS = step1_ks(p, x3), Np = step1_np(p);
  const int n_jt = (K + kTRows - 1) / kTRows;
  const int n_jt_all = (NT + kTRows - 1) / kTRows;
  const int Rt = step1_list_rows(K);
  uint16_t* thi = tbuf;
  uint16_t* tlo = thi + static_cast<size_t>(ni) * p->two_Q * n_jt * Rt * K2;
  uint16_t* ihi = ibuf;
  uint16_t* ilo = ihi + static_cast<size_t>(ni) * p->two_Q * Np * K2;
  {
    const uint16_t* ahi = tall;
    const uint16_t* alo = ahi + static_cast<size_t>(p->two_Q) * n_jt_all * kTRows * K2;
    const long long total = static_cast<long long>(ni) * p->two_Q * n_jt * Rt * (K2 / 8);
    const int grid = static_cast<int>(std::min<long long>((total + 255) / 256, 148LL * 64));
    FTK_LAUNCH(p, kKPackTemplates, s,
               (k_gather_template_tiles<<<grid, 256, 0, s>>>(
                    reinterpret_cast<const uint4*>(ahi), reinterpret_cast<const uint4*>(alo), n_jt_all, list, ni, K,
                    p->two_Q, n_jt, Rt, K2, KS, reinterpret_cast<uint4*>(thi), reinterpret_cast<uint4*>(tlo), x3),
                cudaGetLastError()));
  }
  {
    const long long total = static_cast<long long>(ni) * p->two_Q * Np * (K2 / 8);
    const int grid = static_cast<int>(std::min<long long>((total + 255) / 256, 148LL * 32));
    FTK_LAUNCH(p, kKPackTemplates, s,
               (k_pack_images<<<grid, 256, 0, s>>>(a, ni, p->d_G, p->d_l, p->Hh, p->M, p->two_Q, Np, KS, ihi, ilo, x3),
                cudaGetLastError()));
  }
  return step1_tc_launch(p, x3, thi, tlo, ihi, ilo, ni, K, n_jt, Rt, zhat, s);
}

}  // namespace ftk
