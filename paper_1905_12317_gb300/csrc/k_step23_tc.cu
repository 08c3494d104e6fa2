// Steps 2 and 3 of eq. (fbk3) fused in one tcgen05 kernel, with the best-pose
// epilogue: the DFT over q of Step 2 is computed per pair in shared memory and fed
// straight to the tensor cores, so Z never goes through HBM.
//
//   Z_zeta(gamma_r)        = sum_q Zhat_zeta(q) exp(-2 pi i q r / 2Q)          (Step 2)
//   X(delta_s, gamma_r)    = Re sum_zeta Y'_zeta(delta_s) Z_zeta(gamma_r)       (Step 3)
//
// Roles are swapped with respect to the unfused Step 3: the plan's shift factors
// are the A operand, resident in tensor memory for the CTA's whole life (shift s
// = TMEM lane, K = 2 zeta + {0, 1} = (Re Y', -Im Y') packed two 16-bit values per
// column),
// and Z of one pair is the B operand in shared memory (N = rotations, K = (Re Z,
// Im Z)), so D[s, r] = X(delta_s, gamma_r). This frees the shared memory that the
// shift factors would take and leaves room for two pairs of Z plus the DFT scratch.
//
// Step 2 per pair, 2Q = 12 N1, as a two-factor Cooley-Tukey DFT:
//   q = 12 n1 + n2,  r = k1 + N1 k2,
//   U(k1, n2) = w_2Q^{n2 k1} sum_{n1} Zhat(12 n1 + n2) w_N1^{n1 k1}   (pass A)
//   Z(k1 + N1 k2) = sum_{n2} U(k1, n2) w_12^{n2 k2}                    (pass B)
// Pass A reads Zhat coalesced from HBM (consecutive (n2, zeta) per thread) and
// keeps U in shared memory; pass B rounds Z to the operand mode's 16-bit format (bf16
// hi/lo for BF16x3, one bf16 or fp16 term otherwise) and writes it in the no-swizzle
// K-major core-matrix layout of the B operand.
//
// Warp roles: 0-3 epilogue (one TMEM lane quadrant each; they also load the shift
// factors into TMEM), 4 MMA issuer and TMEM owner, and PW Step-2 producers. BF16x3, where
// the MMAs set the pace: PW = 6 on warps 5-7 and 9-11, two on each SMSP other than the MMA
// warp's, warp 8 idle (measured: 2% faster than 9 placed the same way and 6% faster than
// 11 spread over all four SMSPs; 3 cannot keep up). Single-term modes, whose third of the
// MMAs leaves the producers on the critical path: PW = 11 on warps 5-15.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "fft.cuh"
#include "ftk_internal.h"
#include "tc_engine.h"
#include "tc_ptx.cuh"

namespace ftk {

namespace {

constexpr int kN2 = 12;                   // second DFT factor: 2Q = 12 N1
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
// Threads of a block with PW producer warps: 11 = warps 5-15; 6 = warps 5-7 and 9-11 with
// warp 8 idle (it shares the MMA warp's SMSP).
__host__ __device__ constexpr int threads23(int PW) { return PW == 11 ? 16 * 32 : 12 * 32; }
constexpr uint32_t kTmemCols23 = 512;
constexpr size_t kSmemMax23 = 227 * 1024;

struct Step23Args {
  const float2* zhat;    // [pairs][2Q][Hs] Step-1 output
  const uint32_t* yhi;   // [n_mt * 128][Kpad / 2] packed bf16 pairs, row-major (rows >= N zero)
  const uint32_t* ylo;
  const float2* tw;      // [2Q] exp(-2 pi i t / 2Q)
  int Hh, Hs, Kpad, n_mt, N, IS;
  long long pairs;
  int nj, i0, j0;
  unsigned long long* keys;
  int* err;
  int mode;              // operand mode (tc_ptx.cuh OperandMode)
  int checks;            // 1: the checked kernel variant runs (latches kErrIndex, skips the access)
  const int* list;       // per-image template lists [NI][nj] or NULL
  const float2* shifts;  // [N] shifts in pixels (for windows)
  const float2* center;  // [NI] window centres or NULL
  float window;
  int jbase, key_pos;    // template part of a key's pose index: j - jbase, or the list position jl
};

// 16-bit parts per operand value (hi, lo for BF16x3): shift factors in TMEM, Z in shared memory.
__host__ __device__ constexpr int parts_of(int mode) { return mode == tc::kModeBf16x3 ? 2 : 1; }

// Rotation columns per MMA (N): the widest of 96, 64, 32 that divides 2Q and leaves room
// for two accumulators beside the shift factors in the 512 TMEM columns; 0 if none.
inline int choose_nc(int L, int free_cols) {
  for (int nc : {96, 64, 32})
    if (L % nc == 0 && 2 * nc <= free_cols) return nc;
  return 0;
}

struct Layout23 {
  size_t slot_part, slot, inter_off, tw_off, bar_off, total;
};

__host__ __device__ inline Layout23 layout23(int L, int N1, int IS, int Kpad, int parts) {
  Layout23 o;
  o.slot_part = static_cast<size_t>(L) * Kpad * 2;  // one pair of Z, hi or lo
  o.slot = static_cast<size_t>(parts) * o.slot_part;
  o.inter_off = 2 * o.slot;
  o.tw_off = o.inter_off + static_cast<size_t>(N1) * IS * sizeof(float2);
  o.bar_off = o.tw_off + static_cast<size_t>(L) * sizeof(float2);
  o.total = o.bar_off + 12 * 8 + 16;
  return o;
}

__device__ __forceinline__ unsigned int order_key23(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <int NC>
__device__ __forceinline__ float max_of(const float* v) {
  float t0 = fmaxf(v[0], v[1]), t1 = fmaxf(v[2], v[3]), t2 = fmaxf(v[4], v[5]), t3 = fmaxf(v[6], v[7]);
#pragma unroll
  for (int x = 8; x < NC; x += 8) {
    t0 = fmaxf(t0, fmaxf(v[x], v[x + 1]));
    t1 = fmaxf(t1, fmaxf(v[x + 2], v[x + 3]));
    t2 = fmaxf(t2, fmaxf(v[x + 4], v[x + 5]));
    t3 = fmaxf(t3, fmaxf(v[x + 6], v[x + 7]));
  }
  return fmaxf(fmaxf(t0, t1), fmaxf(t2, t3));
}

// True if the condition holds or checks are compiled out; otherwise latches kErrIndex.
#define FTK_CHECK23(cond) (!kChecks || (cond) || (atomicOr(a.err, kErrIndex), false))

// kChecks: the checked variant (knob "checks"); the default variant has no checks at all.
template <int N1, int NC, bool kChecks, int PW>
__global__ void __launch_bounds__(threads23(PW), 1) k_step23_tc(const Step23Args a) {
  constexpr int kProdWarps = PW;
  constexpr int kProdThreads = PW * 32;
  constexpr int L = kN2 * N1;
  constexpr int n_chunks = L / NC;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int parts = parts_of(a.mode);  // 16-bit parts of the shift factors (TMEM) and of Z (shared memory)
  const int b_parts = parts;
  const Layout23 lay = layout23(L, N1, a.IS, a.Kpad, b_parts);
  float2* inter = reinterpret_cast<float2*>(smem + lay.inter_off);  // U [k1][IS]: (n2, zeta) at n2 Hs + zeta
  float2* tws = reinterpret_cast<float2*>(smem + lay.tw_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  uint64_t* b_full = bars;       // [2] Z of a pair written (producers)
  uint64_t* b_empty = bars + 2;  // [2] MMAs reading that Z done
  uint64_t* d_full = bars + 4;   // [2] accumulator ready
  uint64_t* d_empty = bars + 6;  // [2] accumulator drained
  uint64_t* y_ready = bars + 8;  // shift factors in TMEM
  uint64_t* done_bar = bars + 9;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 10);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* prod_ok = reinterpret_cast<volatile int*>(tmem_slot + 2);
  const int kw = a.Kpad / 2;                    // 32-bit TMEM columns of one part of a shift row
  const int AC = parts * kw;                    // columns of one 128-shift tile (hi, then lo)
  const uint32_t dcol0 = static_cast<uint32_t>(a.n_mt * AC);

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&b_full[s], kProdThreads);
      tc::mbar_init(&b_empty[s], 1);
      tc::mbar_init(&d_full[s], 1);
      tc::mbar_init(&d_empty[s], 128);
    }
    tc::mbar_init(y_ready, 128);
    tc::mbar_init(done_bar, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  for (int e = threadIdx.x; e < L; e += blockDim.x) tws[e] = a.tw[e];
  if (warp == kMmaWarp) tc::tmem_alloc<kTmemCols23>(tmem_slot);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp < kEpiWarps) {
    // ---------------- shift factors -> TMEM, then the epilogue ----------------
    const int quad = warp;
    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
    for (int mt = 0; mt < a.n_mt; ++mt) {
      const size_t row = static_cast<size_t>(mt) * 128 + quad * 32 + lane;
      for (int part = 0; part < parts; ++part) {
        const uint4* src = reinterpret_cast<const uint4*>((part ? a.ylo : a.yhi) + row * kw);
        for (int c0 = 0; c0 < kw; c0 += 8) {
          const uint4 u0 = __ldg(src + c0 / 4), u1 = __ldg(src + c0 / 4 + 1);
          const uint32_t r[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
          if (FTK_CHECK23(mt * AC + part * kw + c0 + 8 <= static_cast<int>(dcol0)))
            tc::tmem_st8(tmem_base + lane_off + mt * AC + part * kw + c0, r);
        }
      }
    }
    tc::tmem_st_wait();
    tc::tc_fence_before();
    tc::mbar_arrive(y_ready);

    const unsigned FULL = 0xFFFFFFFFu;
    int ud = 0;
    bool ok = true;
    for (long long pp = blockIdx.x; pp < a.pairs && ok; pp += gridDim.x) {
      const int il = static_cast<int>(pp / a.nj);
      const int jl = static_cast<int>(pp - static_cast<long long>(il) * a.nj);
      const int i = a.i0 + il;
      const int j = a.list ? __ldg(a.list + static_cast<size_t>(i) * a.nj + jl) : a.j0 + jl;
      const unsigned int jk = static_cast<unsigned int>(a.key_pos ? jl : j - a.jbase);
      const float2 cen = a.center ? a.center[i] : make_float2(0.f, 0.f);
      // the order key of the image's best pose so far: a tile whose maximum is below it
      // cannot take the image's pose, so its argmax search is skipped (keys only grow: a
      // stale value prunes less, never wrongly)
      const unsigned int thr = static_cast<unsigned int>(__ldcg(a.keys + i) >> 32);
      unsigned long long best = 0ull;
      float best_v = -INFINITY;
      for (int c = 0; c < n_chunks && ok; ++c) {
        for (int mt = 0; mt < a.n_mt; ++mt, ++ud) {
          const int sd = ud & 1;
          const bool w = tc::mbar_wait(&d_full[sd], (ud >> 1) & 1, abort_flag, a.err);
          if (!(ok = __all_sync(FULL, w))) break;
          tc::tc_fence_after();
          float v[NC];
          if constexpr (NC == 96) {
            tc::tmem_ld64(tmem_base + lane_off + dcol0 + sd * NC, v);
            tc::tmem_ld32(tmem_base + lane_off + dcol0 + sd * NC + 64, v + 64);
          } else if constexpr (NC == 64) {
            tc::tmem_ld64(tmem_base + lane_off + dcol0 + sd * NC, v);
          } else {
            tc::tmem_ld32(tmem_base + lane_off + dcol0 + sd * NC, v);
          }
          tc::tc_fence_before();
          tc::mbar_arrive(&d_empty[sd]);
          const int s = mt * 128 + quad * 32 + lane;
          bool valid = s < a.N;
          if (valid && a.center) {
            const float2 sh = __ldg(a.shifts + s);
            valid = fabsf(sh.x - cen.x) <= a.window && fabsf(sh.y - cen.y) <= a.window;
          }
          if (!valid) continue;
          const float m = max_of<NC>(v);
          if (m >= best_v && order_key23(m) >= thr) {  // first rotation of the maximum: the smallest pose index
            int xs = 0;
#pragma unroll
            for (int x = NC - 1; x >= 0; --x)
              if (v[x] == m) xs = x;
            const unsigned int idx =
                (jk * L + c * NC + xs) * static_cast<unsigned int>(a.N) + s;
            const unsigned long long key = (static_cast<unsigned long long>(order_key23(m)) << 32) | (0xFFFFFFFFu - idx);
            if (key > best) {
              best = key;
              best_v = m;
            }
          }
        }
      }
      if (!ok) break;
      if (__any_sync(FULL, best != 0ull)) {
#pragma unroll
        for (int off = 16; off; off >>= 1) {
          const unsigned long long o = __shfl_xor_sync(FULL, best, off);
          best = o > best ? o : best;
        }
        if (lane == 0 && best) atomicMax(a.keys + i, best);
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer (the whole warp; one elected lane issues) ----------------
    const unsigned FULL = 0xFFFFFFFFu;
    const uint32_t idesc = tc::idesc_f32acc(128, NC, a.mode);
    const uint32_t sbo = a.Kpad * 16;  // 8-row group stride of the B operand (full K per group)
    // descriptors are advanced by adding (byte offset >> 4) to the start-address field
    // (shared addresses stay below 2^18, so the 14-bit field does not overflow)
    const uint64_t desc0 = tc::smem_desc(tc::smem_u32(smem), 128, sbo);
    const uint64_t lo_step = lay.slot_part >> 4;
    const uint64_t chunk_step = static_cast<uint64_t>((NC / 8) * sbo) >> 4;
    const int ksteps = a.Kpad / 16;
    int ud = 0, it = 0;
    bool ok = __all_sync(FULL, tc::mbar_wait(y_ready, 0, abort_flag, a.err));
    tc::tc_fence_after();
    for (long long pp = blockIdx.x; pp < a.pairs && ok; pp += gridDim.x, ++it) {
      const int slot = it & 1;
      if (!(ok = __all_sync(FULL, tc::mbar_wait(&b_full[slot], (it >> 1) & 1, abort_flag, a.err)))) break;
      tc::tc_fence_after();
      const uint64_t dslot = desc0 + ((slot * lay.slot) >> 4);
      for (int c = 0; c < n_chunks && ok; ++c) {
        const uint64_t dchunk = dslot + c * chunk_step;
        for (int mt = 0; mt < a.n_mt; ++mt, ++ud) {
          const int sd = ud & 1;
          if (!(ok = __all_sync(FULL, tc::mbar_wait(&d_empty[sd], ((ud >> 1) & 1) ^ 1, abort_flag, a.err)))) break;
          tc::tc_fence_after();
          const uint32_t d_tmem = tmem_base + dcol0 + sd * NC;
          // operand ranges of this unit: B rows of the chunk inside the slot, A columns below
          // the accumulators, both accumulators inside the allocation
          const bool unit_ok = FTK_CHECK23(
              (c * (NC / 8) + NC / 8 - 1) * sbo + (ksteps - 1) * 256 + 256 <= lay.slot_part &&
              mt * AC + (parts - 1) * kw + ksteps * 8 <= static_cast<int>(dcol0) &&
              dcol0 + 2 * NC <= kTmemCols23);
          uint32_t ah = tmem_base + mt * AC;
          uint64_t dbh = dchunk;
          if (!unit_ok) {
            // checked run with an operand out of range: no MMA (the accumulator keeps stale values)
          } else if (a.mode == tc::kModeBf16x3) {
#pragma unroll 4
            for (int ks = 0; ks < ksteps; ++ks, ah += 8, dbh += 16)
              tc::mma_bf16x3_ts_warp(d_tmem, ah, ah + kw, dbh, dbh + lo_step, idesc, ks > 0 ? 1u : 0u);
          } else {
            for (int ks = 0; ks < ksteps; ++ks, ah += 8, dbh += 16)
              tc::mma_bf16_ts_warp(d_tmem, ah, dbh, idesc, ks > 0 ? 1u : 0u);
          }
          tc::mma_commit_warp(&d_full[sd]);
        }
      }
      if (!ok) break;
      tc::mma_commit_warp(&b_empty[slot]);
    }
    // wait for every issued MMA before teardown
    tc::mma_commit_warp(done_bar);
    volatile int never = 0;
    tc::mbar_wait(done_bar, 0, &never, a.err, 200000000ull);
  } else if (PW == 11 || warp % 4 != 0) {
    // ---------------- Step 2 producers ----------------
    const int pw = PW == 11 ? warp - 5 : warp - 5 - (warp - 4) / 4;  // 0..PW-1
    const int ptid = pw * 32 + lane;
    {  // zero both Z slots once: the padded K columns (zeta >= Hh) are never written
      uint4* z = reinterpret_cast<uint4*>(smem);
      const int n16 = static_cast<int>(2 * lay.slot / 16);
      for (int e = ptid; e < n16; e += kProdThreads) z[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    const int items_a = kN2 * a.Hs;
    const int n_zb = (a.Hh + 3) / 4;
    constexpr int n_kb = N1 / 8;
    int it = 0;
    for (long long pp = blockIdx.x; pp < a.pairs; pp += gridDim.x, ++it) {
      const int slot = it & 1;
      __syncwarp();
      tc::named_bar_sync(1, kProdThreads);  // the previous pair's reads of U (and the zero fill) are done
      // pass A: Zhat (HBM) -> U (shared), thread = (n2, zeta); the next pair's Zhat
      // is prefetched into L2 meanwhile
      const float2* src = a.zhat + static_cast<size_t>(pp) * L * a.Hs;
      if (ptid == 0 && pp + gridDim.x < a.pairs)
        tc::prefetch_l2(src + static_cast<size_t>(gridDim.x) * L * a.Hs,
                        static_cast<uint32_t>(static_cast<size_t>(L) * a.Hs * sizeof(float2)));
      for (int e = ptid; e < items_a; e += kProdThreads) {
        const int n2 = e / a.Hs;
        const int z = e - n2 * a.Hs;
        if (z >= a.Hh) continue;
        if (!FTK_CHECK23(e < a.IS && static_cast<size_t>(pp) * L * a.Hs + static_cast<size_t>(kN2 * (N1 - 1)) * a.Hs + e <
                                         static_cast<size_t>(a.pairs) * L * a.Hs))
          continue;
        float2 x[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = __ldg(src + static_cast<size_t>(kN2 * n1) * a.Hs + e);
        dft_reg<N1>(x, tws, L / N1);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) inter[k1 * a.IS + e] = k1 ? cmul(x[k1], tws[n2 * k1]) : x[k1];
      }
      if (ptid == 0) *prod_ok = tc::mbar_wait(&b_empty[slot], ((it >> 1) & 1) ^ 1, abort_flag, a.err) ? 1 : 0;
      __syncwarp();
      tc::named_bar_sync(1, kProdThreads);  // U complete; the slot is free
      if (!*prod_ok) break;
      // pass B: U -> Z (bf16 hi/lo, B-operand layout), warp task = 8 k1 x 4 zeta
      uint8_t* base_hi = smem + slot * lay.slot;
      uint8_t* base_lo = base_hi + lay.slot_part;
      for (int t = pw; t < n_kb * n_zb; t += kProdWarps) {
        const int kb = t % n_kb, zb = t / n_kb;
        const int k1 = kb * 8 + (lane & 7);
        const int z = zb * 4 + (lane >> 3);
        if (z >= a.Hh) continue;
        float2 v[kN2];
#pragma unroll
        if (!FTK_CHECK23(k1 * a.IS + (kN2 - 1) * a.Hs + z < N1 * a.IS &&
                         static_cast<size_t>(((k1 + N1 * (kN2 - 1)) >> 3) * 16 * a.Kpad + 128 * (z >> 2) + 128) <=
                             lay.slot_part))
          continue;
        for (int n2 = 0; n2 < kN2; ++n2) v[n2] = inter[k1 * a.IS + n2 * a.Hs + z];
        dft_reg<kN2>(v, tws, L / kN2);
#pragma unroll
        for (int k2 = 0; k2 < kN2; ++k2) {
          const int r = k1 + N1 * k2;
          const uint32_t off = static_cast<uint32_t>((r >> 3) * 16 * a.Kpad + (z >> 2) * 128 + (r & 7) * 16 + (z & 3) * 4);
          uint32_t hi, lo;
          tc::pack2(v[k2].x, v[k2].y, a.mode, hi, lo);
          *reinterpret_cast<uint32_t*>(base_hi + off) = hi;
          if (b_parts == 2) *reinterpret_cast<uint32_t*>(base_lo + off) = lo;
        }
      }
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(&b_full[slot]);
    }
  }

  __syncwarp();  // the single-lane roles rejoin their warps
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == kMmaWarp) tc::tmem_dealloc<kTmemCols23>(tmem_base);
}

int n1_of(int L) { return L == 96 ? 8 : (L == 192 ? 16 : 0); }

int inter_stride(int Hs) {
  int IS = kN2 * Hs;
  // = 2 mod 16 (8-byte words): the 16 lanes of each half-warp of a pass-B read (8 k1 x
  // 2 zeta) fall on 16 different bank pairs
  IS += ((2 - IS % 16) + 16) % 16;
  return IS;
}

template <int N1, int NC>
ftk_status launch23(ftk_plan_s* p, const Step23Args& args, cudaStream_t s) {
  const Layout23 lay = layout23(kN2 * N1, N1, args.IS, args.Kpad, parts_of(args.mode));
  const bool x3 = args.mode == tc::kModeBf16x3;
  auto kernel = args.checks ? (x3 ? k_step23_tc<N1, NC, true, 6> : k_step23_tc<N1, NC, true, 11>)
                            : (x3 ? k_step23_tc<N1, NC, false, 6> : k_step23_tc<N1, NC, false, 11>);
  const int threads = threads23(x3 ? 6 : 11);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(lay.total));
  if (e != cudaSuccess) return FTK_ERR_CUDA;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = static_cast<int>(std::min<long long>(args.pairs, nsm));
  FTK_LAUNCH(p, kKStep23Tc, s,
             (kernel<<<grid, threads, lay.total, s>>>(args), cudaGetLastError()));
  return FTK_OK;
}

}  // namespace

namespace {
int step23_nc(const ftk_plan_s* p, int mode) {
  const int free_cols = static_cast<int>(kTmemCols23) - p->tc.n_mt * parts_of(mode) * (p->tc.Kpad / 2);
  return choose_nc(p->two_Q, free_cols);
}
}  // namespace

bool step23_supported(const ftk_plan_s* p, int precision) {
  if (p->tune.step23 == 0 || !p->tc.d_Yrhi || p->n_rot != p->two_Q) return false;
  const int L = p->two_Q;
  const int N1 = n1_of(L);
  if (!N1) return false;
  const int mode = op_mode(precision);
  if (!step23_nc(p, mode)) return false;
  const int Hs = (p->Hh + 1) & ~1;
  return layout23(L, N1, inter_stride(Hs), p->tc.Kpad, parts_of(mode)).total <= kSmemMax23;
}

ftk_status step23_run(ftk_plan_s* p, int precision, const float2* zhat, long long pairs, int nj, int i0, int j0,
                      unsigned long long* keys, const int* list, const float2* center, float window, int jbase,
                      int key_pos, cudaStream_t s) {
  if (!step23_supported(p, precision)) return FTK_ERR_UNSUPPORTED;
  if (pairs <= 0) return FTK_OK;
  Step23Args a;
  a.zhat = zhat;
  const int mode = op_mode(precision);
  a.yhi = reinterpret_cast<const uint32_t*>(mode == tc::kModeF16 ? p->tc.d_Yr16 : p->tc.d_Yrhi);
  a.ylo = reinterpret_cast<const uint32_t*>(p->tc.d_Yrlo);
  a.tw = p->d_tw;
  a.Hh = p->Hh;
  a.Hs = (p->Hh + 1) & ~1;
  a.Kpad = p->tc.Kpad;
  a.n_mt = p->tc.n_mt;
  a.N = p->N;
  a.IS = inter_stride(a.Hs);
  a.pairs = pairs;
  a.nj = nj;
  a.i0 = i0;
  a.j0 = j0;
  a.keys = keys;
  a.err = p->d_err;
  a.mode = mode;
  a.checks = p->tune.checks;
  a.list = list;
  a.shifts = p->d_shifts;
  a.center = center;
  a.window = window;
  a.jbase = jbase;
  a.key_pos = key_pos;
  const int nc = step23_nc(p, mode);
  switch (n1_of(p->two_Q) * 1000 + nc) {
    case 8096: return launch23<8, 96>(p, a, s);
    case 8032: return launch23<8, 32>(p, a, s);
    case 16096: return launch23<16, 96>(p, a, s);
    case 16064: return launch23<16, 64>(p, a, s);
    case 16032: return launch23<16, 32>(p, a, s);
    default: return FTK_ERR_UNSUPPORTED;
  }
}

}  // namespace ftk
