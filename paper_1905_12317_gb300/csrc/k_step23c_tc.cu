// Steps 2 and 3 of eq. (fbk3) fused for 2Q = 128 R (R = 2, 3, 4; 2Q = 384 on the n = 128
// grid) over a cluster of C CTAs, with the best-pose epilogue. Z never goes through HBM.
//
//   Z_zeta(gamma_r)        = sum_q Zhat_zeta(q) exp(-2 pi i q r / 2Q)          (Step 2)
//   X(delta_s, gamma_r)    = Re sum_zeta Y'_zeta(delta_s) Z_zeta(gamma_r)       (Step 3)
//
// Step 3 is the GEMM of the unfused tensor-core kernel: D[(pair, r), s] = sum_k A[(pair, r), k]
// B[s, k] with A = (Re Z, Im Z) and B = (Re Y', -Im Y') (Y' = c_l Y), K = 2 zeta + {0, 1}. The
// shifts are split into C groups of G (the plan's Step-3 groups); CTA `rank` of a cluster holds
// group `rank` of B in shared memory for its whole life, so each MMA has the wide N = G.
//
// A is produced on chip, one 128-row tile (128 rotations of one pair) at a time, split along K
// into slices of 16 zeta (32 K columns). The slices of a tile are produced by the CTAs of the
// cluster in turn (slice s by CTA s mod C) and each is sent, by bulk copies over the cluster's
// shared-memory window, into the same ring slot of every CTA of the cluster; a CTA's MMAs
// release a slot by a multicast commit on the producing CTA's barrier. So the DFT over q of
// a pair is computed once per cluster, and every CTA multiplies all of it with its shifts.
//
// Rotation tiles: r = R r' + c, r' = 0..127, c = 0..R-1 (one tile per c). With q = q' + 128 b,
//   Z(R r' + c) = sum_{q'} w_128^{q' r'} v_c(q'),  v_c(q') = w_2Q^{q' c} sum_b Zhat(q' + 128 b) w_R^{b c}
// (a radix-R decimation-in-frequency step, then a length-128 DFT per zeta). Row r' of the tile
// is rotation R r' + c.
//
// Warp roles: 0 MMA issuer and TMEM owner (also loads B), 1 idle, 2-9 epilogue (two warps per
// TMEM lane quadrant, the first on the accumulator's first columns, the second on the rest),
// 10-17 producers (v_c into shared memory, then one warp FFT per zeta). A producer thread loads
// its Zhat values once per pair (all R rotation tiles of a pair use the same ones) and issues
// the next pair's loads before the FFT of the pair's last tile, so their latency is hidden.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "fft.cuh"
#include "ftk_internal.h"
#include "tc_engine.h"
#include "tc_ptx.cuh"

namespace ftk {

namespace {

constexpr int kTileRows = 128;  // rotations per A tile (MMA M)
constexpr int kSliceK = 32;     // K columns per slice (16 zeta)
constexpr int kSliceZ = kSliceK / 2;
constexpr int kProducers = 8;   // producer warps
constexpr int kEpiWarps = 8;    // epilogue warps: two per TMEM lane quadrant, each on part of the columns
constexpr int kFirstEpi = 2;
constexpr int kFirstProducer = kFirstEpi + kEpiWarps;
constexpr int kThreadsC = (kFirstProducer + kProducers) * 32;
constexpr int kVStride = kSliceZ + 1;  // complex row stride of the v_c scratch [128 q'][16 zeta]
constexpr uint32_t kTmemColsC = 512;
constexpr size_t kSmemMaxC = 227 * 1024;

struct Step23cArgs {
  const float2* zhat;    // [pairs][2Q][Hs] Step-1 output
  const uint16_t* yhi;   // [n_groups * G][Kpad] the Step-3 B operand (core-matrix layout), bf16 or fp16
  const uint16_t* ylo;   // its bf16 residuals (BF16x3)
  const float2* tw;      // [2Q] exp(-2 pi i t / 2Q)
  int L;                 // 2Q
  int Hh, Hs, Kpad, n_slices, G, N;
  long long pairs;
  int nj, i0, j0;
  int jbase, key_pos;    // template part of a key's pose index: j - jbase, or the list position jl
  unsigned long long* keys;
  int* err;
  int mode;
  const int* list;       // per-image template lists [NI][nj] or NULL
  const float2* shifts;  // [N] shifts in pixels (for windows)
  const float2* center;  // [NI] window centres or NULL
  float window;
};

struct LayoutC {
  size_t y_part, slot_part, slot, ring_off, stg_off, v_off, tw_off, tw128_off, bar_off, total;
};

__host__ __device__ inline LayoutC layout_c(int G, int Kpad, int n_slices, int parts, int L) {
  LayoutC o;
  o.y_part = static_cast<size_t>(G) * Kpad * 2;
  o.slot_part = static_cast<size_t>(kTileRows) * kSliceK * 2;
  o.slot = static_cast<size_t>(parts) * o.slot_part;
  o.ring_off = static_cast<size_t>(parts) * o.y_part;
  o.stg_off = o.ring_off + static_cast<size_t>(n_slices) * o.slot;
  o.v_off = o.stg_off + 2 * o.slot;
  o.tw_off = o.v_off + static_cast<size_t>(kTileRows) * kVStride * sizeof(float2);
  o.tw128_off = o.tw_off + static_cast<size_t>(L) * sizeof(float2);
  o.bar_off = o.tw128_off + kTileRows * sizeof(float2);
  o.total = o.bar_off + static_cast<size_t>(2 * n_slices + 6) * 8 + 16;
  return o;
}

__device__ __forceinline__ unsigned int order_key_c(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float max_of64(const float* v) {
  float t0 = fmaxf(v[0], v[1]), t1 = fmaxf(v[2], v[3]), t2 = fmaxf(v[4], v[5]), t3 = fmaxf(v[6], v[7]);
#pragma unroll
  for (int x = 8; x < 64; x += 8) {
    t0 = fmaxf(t0, fmaxf(v[x], v[x + 1]));
    t1 = fmaxf(t1, fmaxf(v[x + 2], v[x + 3]));
    t2 = fmaxf(t2, fmaxf(v[x + 4], v[x + 5]));
    t3 = fmaxf(t3, fmaxf(v[x + 6], v[x + 7]));
  }
  return fmaxf(fmaxf(t0, t1), fmaxf(t2, t3));
}

// Element offset of (row, k) in one part of an A slice: no-swizzle K-major core matrices,
// 8-row groups of kSliceK elements, the K core matrices of a group contiguous.
__device__ __forceinline__ uint32_t slice_off(int row, int k) {
  return static_cast<uint32_t>((row >> 3) * 8 * kSliceK + (k >> 3) * 64 + (row & 7) * 8 + (k & 7));
}

// kWin: shift windows (per-image centres) are tested in the epilogue; without, no window code.
template <int R, bool kWin>
__global__ void __launch_bounds__(kThreadsC, 1) k_step23c_tc(const Step23cArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int parts = tc::mode_split(a.mode) ? 2 : 1;
  const int ns = a.n_slices;
  const LayoutC lay = layout_c(a.G, a.Kpad, ns, parts, a.L);
  const uint32_t rank = tc::cluster_ctarank();
  const uint32_t C = tc::cluster_nctarank();
  const long long cid = tc::cluster_id_x(), ncl = tc::nclusters_x();
  uint8_t* ys = smem;
  uint8_t* ring = smem + lay.ring_off;
  uint8_t* stg = smem + lay.stg_off;
  float2* vs = reinterpret_cast<float2*>(smem + lay.v_off);
  float2* tws = reinterpret_cast<float2*>(smem + lay.tw_off);
  float2* tw128 = reinterpret_cast<float2*>(smem + lay.tw128_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  uint64_t* y_full = bars;
  uint64_t* full = bars + 1;               // [ns] slot s holds the current tile's slice s
  uint64_t* peer_empty = full + ns;        // [ns] slot s released by all C CTAs (this CTA produces s)
  uint64_t* d_full = peer_empty + ns;      // [2] accumulator ready
  uint64_t* d_empty = d_full + 2;          // [2] accumulator drained
  uint64_t* done_bar = d_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* prod_ok = reinterpret_cast<volatile int*>(tmem_slot + 2);
  const uint32_t slot_bytes = static_cast<uint32_t>(lay.slot);
  const unsigned FULL = 0xFFFFFFFFu;

  if (threadIdx.x == 0) {
    tc::mbar_init(y_full, 1);
    for (int s = 0; s < ns; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&peer_empty[s], C);
    }
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&d_full[s], 1);
      tc::mbar_init(&d_empty[s], kEpiWarps * 32);
    }
    tc::mbar_init(done_bar, 1);
    for (int s = 0; s < ns; ++s) tc::mbar_arrive_expect_tx(&full[s], slot_bytes);  // phase 0 of every slot
    *abort_flag = 0;
    *prod_ok = 1;
    tc::fence_barrier_init();
  }
  for (int e = threadIdx.x; e < a.L; e += blockDim.x) tws[e] = a.tw[e];
  for (int e = threadIdx.x; e < kTileRows; e += blockDim.x) tw128[e] = a.tw[e * R];  // w_128^e = w_2Q^{R e}
  if (warp == 0) tc::tmem_alloc<kTmemColsC>(tmem_slot);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  // every CTA of the cluster has initialized its barriers before any copy or arrival reaches it
  tc::cluster_sync();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- B operand load, then the MMA issuer (one elected lane issues) ----------------
    if (lane == 0) {
      const size_t goff = static_cast<size_t>(rank) * a.G * a.Kpad;
      tc::mbar_arrive_expect_tx(y_full, static_cast<uint32_t>(parts * lay.y_part));
      tc::bulk_g2s(ys, a.yhi + goff, static_cast<uint32_t>(lay.y_part), y_full);
      if (parts == 2) tc::bulk_g2s(ys + lay.y_part, a.ylo + goff, static_cast<uint32_t>(lay.y_part), y_full);
    }
    __syncwarp();
    const uint32_t idesc = tc::idesc_f32acc(kTileRows, a.G, a.mode);
    const uint64_t dy0 = tc::smem_desc(tc::smem_u32(ys), 128, a.Kpad * 16);
    const uint64_t dr0 = tc::smem_desc(tc::smem_u32(ring), 128, kSliceK * 16);
    const uint64_t y_lo_step = lay.y_part >> 4, a_lo_step = lay.slot_part >> 4;
    const bool split = tc::mode_split(a.mode);
    bool ok = __all_sync(FULL, tc::mbar_wait(y_full, 0, abort_flag, a.err));
    tc::tc_fence_after();
    int ud = 0;
    for (long long pp = cid; pp < a.pairs && ok; pp += ncl) {
      for (int c = 0; c < R && ok; ++c, ++ud) {
        const int sd = ud & 1;
        if (!(ok = __all_sync(FULL, tc::mbar_wait(&d_empty[sd], ((ud >> 1) & 1) ^ 1, abort_flag, a.err)))) break;
        tc::tc_fence_after();
        const uint32_t d_tmem = tmem_base + sd * a.G;
        for (int s = 0; s < ns; ++s) {
          if (!(ok = __all_sync(FULL, tc::mbar_wait(&full[s], ud & 1, abort_flag, a.err)))) break;
          tc::tc_fence_after();
          uint64_t dah = dr0 + ((static_cast<uint64_t>(s) * slot_bytes) >> 4);
          uint64_t dbh = dy0 + static_cast<uint64_t>(s * (kSliceK / 16)) * 16;  // two core matrices per k-step
#pragma unroll
          for (int kk = 0; kk < kSliceK / 16; ++kk, dah += 16, dbh += 16) {
            const uint32_t acc = (s > 0 || kk > 0) ? 1u : 0u;
            if (split)
              tc::mma_bf16x3_ss_warp(d_tmem, dah, dah + a_lo_step, dbh, dbh + y_lo_step, idesc, acc);
            else
              tc::mma_bf16_ss_warp(d_tmem, dah, dbh, idesc, acc);
          }
          // the slot is free here once these MMAs complete: tell the CTA that produces it
          tc::mma_commit_multicast_warp(&peer_empty[s], static_cast<uint16_t>(1u << (s % C)));
          if (lane == 0) tc::mbar_arrive_expect_tx(&full[s], slot_bytes);  // arm the slot's next phase
          __syncwarp();
        }
        if (!ok) break;
        tc::mma_commit_warp(&d_full[sd]);
      }
    }
    // wait for every issued MMA before teardown
    tc::mma_commit_warp(done_bar);
    volatile int never = 0;
    tc::mbar_wait(done_bar, 0, &never, a.err, 200000000ull);
  } else if (warp >= kFirstEpi && warp < kFirstProducer) {
    // ---------------- epilogue: per tile, the per-image maximum over this CTA's shifts ----------------
    const int quad = warp & 3;
    const int row = quad * 32 + lane;  // tile row = r'
    const int g0 = static_cast<int>(rank) * a.G;
    // columns [cb, ce) of the accumulator: the first warp of a quadrant takes the first half
    // rounded up to 64, the second the rest
    const int half = (warp - kFirstEpi) / 4;
    const int cmid = min(a.G, (a.G / 2 + 63) / 64 * 64);
    const int cb = half ? cmid : 0, ce = half ? a.G : cmid;
    int ud = 0;
    bool ok = true;
    for (long long pp = cid; pp < a.pairs && ok; pp += ncl) {
      const int il = static_cast<int>(pp / a.nj);
      const int jl = static_cast<int>(pp - static_cast<long long>(il) * a.nj);
      const int i = a.i0 + il;
      const int j = a.list ? __ldg(a.list + static_cast<size_t>(i) * a.nj + jl) : a.j0 + jl;
      const unsigned int jk = static_cast<unsigned int>(a.key_pos ? jl : j - a.jbase);
      const float2 cen = kWin ? a.center[i] : make_float2(0.f, 0.f);
      // the order key of the image's best pose so far: a row whose maximum is below it cannot
      // take the image's pose, so it skips the argmax search and the atomic (keys only grow:
      // a stale value prunes less, never wrongly)
      const unsigned int thr = static_cast<unsigned int>(__ldcg(a.keys + i) >> 32);
      for (int c = 0; c < R; ++c, ++ud) {
        const int sd = ud & 1;
        if (!(ok = __all_sync(FULL, tc::mbar_wait(&d_full[sd], (ud >> 1) & 1, abort_flag, a.err)))) break;
        tc::tc_fence_after();
        const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quad * 32) << 16) + sd * a.G;
        float best_v = -INFINITY;
        int best_s = 0;
        if (cb >= ce) {  // no columns for this warp (G <= 64): it still releases the accumulator
          tc::tc_fence_before();
          tc::mbar_arrive(&d_empty[sd]);
        }
        for (int c0 = cb; c0 < ce;) {
          const int w = ce - c0 >= 64 ? 64 : (ce - c0 >= 32 ? 32 : 16);
          float v[64];
          if (w == 64) tc::tmem_ld64(taddr + c0, v);
          else if (w == 32) tc::tmem_ld32(taddr + c0, v);
          else tc::tmem_ld16(taddr + c0, v);
          if (c0 + w >= ce) {  // the accumulator is free once its last columns are in registers
            tc::tc_fence_before();
            tc::mbar_arrive(&d_empty[sd]);
          }
          // columns past this load, past the last shift or outside the window do not count;
          // the tests are uniform across the warp (the column is the shift), so no divergence
          const int nvalid = min(w, a.N - (g0 + c0));
#pragma unroll
          for (int x = 0; x < 64; ++x) {
            bool in = x < nvalid;
            if (kWin && in) {
              const float2 sh = __ldg(a.shifts + g0 + c0 + x);
              in = fabsf(sh.x - cen.x) <= a.window && fabsf(sh.y - cen.y) <= a.window;
            }
            v[x] = in ? v[x] : -INFINITY;
          }
          const float m = max_of64(v);
          if (m > best_v) {  // the first column of the maximum: the smallest shift index
            best_v = m;
            if (order_key_c(m) >= thr) {
              int xs = 0;
#pragma unroll
              for (int x = 63; x >= 0; --x) xs = v[x] == m ? x : xs;
              best_s = g0 + c0 + xs;
            }
          }
          c0 += w;
        }
        unsigned long long key = 0ull;
        if (best_v > -INFINITY && order_key_c(best_v) >= thr) {  // best_s holds best_v's shift
          const unsigned int r = static_cast<unsigned int>(R * row + c);
          const unsigned int idx = (jk * a.L + r) * static_cast<unsigned int>(a.N) + best_s;
          key = (static_cast<unsigned long long>(order_key_c(best_v)) << 32) | (0xFFFFFFFFu - idx);
        }
        if (__any_sync(FULL, key != 0ull)) {
#pragma unroll
          for (int off = 16; off; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(FULL, key, off);
            key = o > key ? o : key;
          }
          if (lane == 0 && key) atomicMax(a.keys + i, key);
        }
      }
    }
  } else if (warp >= kFirstProducer && static_cast<int>(rank) < ns) {
    // ---------------- producers: slice s = rank of every tile (at most one per tile) ----------------
    const int pw = warp - kFirstProducer;
    const int pt = pw * 32 + lane;
    const int zl = pt & (kSliceZ - 1), qs = pt / kSliceZ;  // phase A: (q' = qs + 16 it, zeta zl)
    constexpr int kQStep = kProducers * 32 / kSliceZ;       // 16
    constexpr int kIt = kTileRows / kQStep;                  // 8
    const int s = static_cast<int>(rank);
    const int z = s * kSliceZ + zl;
    const size_t pstride = static_cast<size_t>(a.L) * a.Hs;
    // Zhat(q' + 128 b, z) of the current pair, q' = qs + 16 it: the same for every tile of the pair
    float2 x[kIt][R];
    auto load_pair = [&](long long pq) {
      const float2* src = a.zhat + static_cast<size_t>(pq) * pstride;
#pragma unroll
      for (int it = 0; it < kIt; ++it)
#pragma unroll
        for (int b = 0; b < R; ++b)
          x[it][b] = (z < a.Hh && pq < a.pairs)
                         ? __ldg(src + static_cast<size_t>(qs + kQStep * it + kTileRows * b) * a.Hs + z)
                         : make_float2(0.f, 0.f);
    };
    load_pair(cid);
    int ud = 0;
    bool ok = true;
    for (long long pp = cid; pp < a.pairs && ok; pp += ncl) {
      if (pt == 0 && rank == 0 && pp + ncl < a.pairs)  // the cluster's next pair into L2
        tc::prefetch_l2(a.zhat + static_cast<size_t>(pp + ncl) * pstride,
                        static_cast<uint32_t>(pstride * sizeof(float2)));
      for (int c = 0; c < R; ++c, ++ud) {
        // phase A: v_c(q', zeta) into shared memory (the previous task's phase-B reads are done)
        __syncwarp();
        tc::named_bar_sync(1, kProducers * 32);
        if (!*prod_ok) {
          ok = false;
          break;
        }
#pragma unroll
        for (int it = 0; it < kIt; ++it) {
          const int qp = qs + kQStep * it;
          float2 acc = x[it][0];
#pragma unroll
          for (int b = 1; b < R; ++b) acc = c ? cadd(acc, cmul(x[it][b], tws[(kTileRows * b * c) % a.L])) : cadd(acc, x[it][b]);
          if (c) acc = cmul(acc, tws[(qp * c) % a.L]);
          vs[qp * kVStride + zl] = acc;
        }
        if (c == R - 1) load_pair(pp + ncl);  // the next pair's loads, in flight during this FFT
        __syncwarp();
        tc::named_bar_sync(1, kProducers * 32);
        // phase B: one length-128 DFT per zeta (two per warp), rounded to the operand format
        // and written in the slice layout (K = 2 zeta + {Re, Im}) of staging buffer ud & 1
        uint8_t* st = stg + (ud & 1) * static_cast<size_t>(slot_bytes);
        {
          float2 x0[4], x1[4];
          const int za = 2 * pw;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            x0[k] = vs[(lane + 32 * k) * kVStride + za];
            x1[k] = vs[(lane + 32 * k) * kVStride + za + 1];
          }
          warp_fft<kTileRows>(x0, tw128);
          warp_fft<kTileRows>(x1, tw128);
          const int br = static_cast<int>(__brev(static_cast<unsigned>(lane)) >> 27);
#pragma unroll
          for (int f2 = 0; f2 < 4; ++f2) {
            const int rr = f2 + 4 * br;  // r' of lane's f2-th output
            uint32_t h0, l0, h1, l1;
            tc::pack2(x0[f2].x, x0[f2].y, a.mode, h0, l0);
            tc::pack2(x1[f2].x, x1[f2].y, a.mode, h1, l1);
            const uint32_t off = slice_off(rr, 2 * za) * 2;  // bytes; 2 za, 2 za + 1, ... + 3: 8 bytes
            *reinterpret_cast<uint2*>(st + off) = make_uint2(h0, h1);
            if (parts == 2) *reinterpret_cast<uint2*>(st + lay.slot_part + off) = make_uint2(l0, l1);
          }
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        tc::named_bar_sync(1, kProducers * 32);
        if (pt == 0) {
          // slot s is free in every CTA once all C CTAs released the previous tile's slice s
          const bool w = tc::mbar_wait(&peer_empty[s], (ud & 1) ^ 1, abort_flag, a.err);
          if (w) {
            const uint32_t dst = tc::smem_u32(ring + static_cast<size_t>(s) * slot_bytes);
            const uint32_t bar = tc::smem_u32(&full[s]);
            for (uint32_t d = 0; d < C; ++d)
              tc::bulk_s2cluster(tc::mapa_shared(dst, d), st, slot_bytes, tc::mapa_shared(bar, d));
          } else {
            *prod_ok = 0;
          }
        }
      }
    }
  }

  __syncwarp();  // the single-lane roles rejoin their warps
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc<kTmemColsC>(tmem_base);
  // no CTA leaves while a peer may still copy into its shared memory or arrive on its barriers
  tc::cluster_sync();
}

int radix_of(int L) { return (L % kTileRows == 0 && L / kTileRows >= 2 && L / kTileRows <= 4) ? L / kTileRows : 0; }

template <int R, bool kWin>
cudaError_t cluster_config(const ftk_plan_s* p, size_t smem, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr) {
  auto kernel = k_step23c_tc<R, kWin>;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int C = p->tc.n_groups;
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3(static_cast<unsigned>(C), 1, 1);
  cfg->blockDim = dim3(kThreadsC, 1, 1);
  cfg->dynamicSmemBytes = smem;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(C);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  return cudaSuccess;
}

// Clusters of the plan's group count that can run at once (0 if none).
template <int R>
int max_clusters(const ftk_plan_s* p, size_t smem) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  // the windowed variant is configured too, so that either can be launched afterwards
  if (cluster_config<R, true>(p, smem, &cfg, attr) != cudaSuccess ||
      cluster_config<R, false>(p, smem, &cfg, attr) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_step23c_tc<R, false>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int max_clusters_r(const ftk_plan_s* p, size_t smem) {
  switch (radix_of(p->two_Q)) {
    case 2: return max_clusters<2>(p, smem);
    case 3: return max_clusters<3>(p, smem);
    case 4: return max_clusters<4>(p, smem);
    default: return 0;
  }
}

size_t smem_c(const ftk_plan_s* p, int mode) {
  const int parts = tc::mode_split(mode) ? 2 : 1;
  return layout_c(p->tc.G, p->tc.Kpad, p->tc.Kpad / kSliceK, parts, p->two_Q).total;
}

template <int R, bool kWin>
ftk_status launch_c(ftk_plan_s* p, const Step23cArgs& args, int n_clusters, cudaStream_t s) {
  const size_t smem = layout_c(args.G, args.Kpad, args.n_slices, tc::mode_split(args.mode) ? 2 : 1, args.L).total;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  if (cluster_config<R, kWin>(p, smem, &cfg, attr) != cudaSuccess) return FTK_ERR_CUDA;
  cfg.gridDim = dim3(static_cast<unsigned>(p->tc.n_groups * n_clusters), 1, 1);
  cfg.stream = s;
  FTK_LAUNCH(p, kKStep23cTc, s, cudaLaunchKernelEx(&cfg, k_step23c_tc<R, kWin>, args));
  return FTK_OK;
}

}  // namespace

bool step23c_supported(ftk_plan_s* p, int precision) {
  if (p->tune.step23 == 0 || p->tune.cluster23 == 0 || !p->tc.d_Yhi || p->n_rot != p->two_Q) return false;
  if (!radix_of(p->two_Q) || p->tc.Kpad % kSliceK != 0) return false;
  if (p->tc.n_groups < 2 || p->tc.n_groups > 8 || p->tc.G % 16 != 0) return false;
  // each CTA produces at most one slice per tile: a staging buffer is then reused only after
  // the slot it last filled was released (the producer waits for that before its next copy)
  if (p->tc.Kpad / kSliceK > p->tc.n_groups) return false;
  const int mode = op_mode(precision);
  const size_t smem = smem_c(p, mode);
  if (smem > kSmemMaxC) return false;
  int& cached = p->tc.max_clusters[mode];
  if (cached < 0) cached = max_clusters_r(p, smem);
  return cached > 0;
}

ftk_status step23c_run(ftk_plan_s* p, int precision, const float2* zhat, long long pairs, int nj, int i0, int j0,
                       unsigned long long* keys, const int* list, const float2* center, float window, int jbase,
                       int key_pos, cudaStream_t s) {
  if (!step23c_supported(p, precision)) return FTK_ERR_UNSUPPORTED;
  if (pairs <= 0) return FTK_OK;
  const int mode = op_mode(precision);
  Step23cArgs a;
  a.zhat = zhat;
  a.yhi = mode == tc::kModeF16 ? p->tc.d_Yh16 : p->tc.d_Yhi;
  a.ylo = p->tc.d_Ylo;
  a.tw = p->d_tw;
  a.L = p->two_Q;
  a.Hh = p->Hh;
  a.Hs = (p->Hh + 1) & ~1;
  a.Kpad = p->tc.Kpad;
  a.n_slices = p->tc.Kpad / kSliceK;
  a.G = p->tc.G;
  a.N = p->N;
  a.pairs = pairs;
  a.nj = nj;
  a.i0 = i0;
  a.j0 = j0;
  a.jbase = jbase;
  a.key_pos = key_pos;
  a.keys = keys;
  a.err = p->d_err;
  a.mode = mode;
  a.list = list;
  a.shifts = p->d_shifts;
  a.center = center;
  a.window = window;
  const int ncl = static_cast<int>(std::min<long long>(pairs, p->tc.max_clusters[mode]));
  const bool win = center != nullptr;
  switch (radix_of(p->two_Q) * 2 + (win ? 1 : 0)) {
    case 4: return launch_c<2, false>(p, a, ncl, s);
    case 5: return launch_c<2, true>(p, a, ncl, s);
    case 6: return launch_c<3, false>(p, a, ncl, s);
    case 7: return launch_c<3, true>(p, a, ncl, s);
    case 8: return launch_c<4, false>(p, a, ncl, s);
    case 9: return launch_c<4, true>(p, a, ncl, s);
    default: return FTK_ERR_UNSUPPORTED;
  }
}

}  // namespace ftk
