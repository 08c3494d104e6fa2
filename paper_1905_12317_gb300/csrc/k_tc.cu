// Tensor-core (tcgen05) pair engine for sm_103a: Step 2 packing and Step 3.
//
// Step 3 of eq. (fbk3) is the dominant contraction:
//   X(delta_s, gamma_r) = Re sum_{zeta: l >= 0} c_l Y_zeta(delta_s) Z_zeta(gamma_r)
// written as a real GEMM  D[(pair, r), s] = sum_k A[(pair, r), k] B[s, k]  with
// k = 2 zeta + {0, 1}:  A = (Re Z, Im Z),  B = (Re Y', -Im Y')  (Y' = c_l Y).
// A (produced per pair by the DFT of Step 2) and B (fixed by the plan) are stored
// in the no-swizzle K-major "core matrix" layout of tcgen05 (8 rows x 16 bytes per
// core matrix; within an 8-row group the K core matrices are contiguous), so any
// run of whole 8-row groups is one contiguous block moved by one bulk async copy.
//
// The shifts are split into n_groups groups of G (MMA N = G <= 256). A CTA owns
// one group for its whole life: its slice of B stays resident in shared memory,
// and it streams 128-row A tiles through a double buffer, with two TMEM
// accumulators so that the epilogue of one tile overlaps the MMAs of the next.
//
// BF16x3: each FP32 operand x is split as x_hi = bf16(x), x_lo = bf16(x - x_hi);
// D accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 (TMEM).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fft.cuh"
#include "ftk_internal.h"
#include "tc_engine.h"
#include "tc_ptx.cuh"

namespace ftk {

namespace {

constexpr int kRows = 128;  // rows of an A tile (MMA M)
constexpr int kTmemCols = 512;
constexpr size_t kSmemBudget = 220 * 1024;

__host__ __device__ inline size_t canon_off(int row, int k, int Kpad) {
  // element offset of (row, k) inside a block whose rows start at 0
  return static_cast<size_t>(row >> 3) * 8 * Kpad + static_cast<size_t>(k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

// K-slice width of the A operand of Step 3: tiles are stored slice by slice,
// [tile][slice][128 rows][KS], so that each K-slice is one contiguous block. The widest
// that divides Kpad: with 64-wide slices the MMA warp waits once per 12 MMAs (BF16x3)
// instead of 6, which made Step 3 2% faster at n = 128.
__host__ __device__ inline int a_slice_width(int Kpad) { return (Kpad % 64 == 0) ? 64 : (Kpad % 32 == 0) ? 32 : 16; }

__host__ __device__ inline size_t a_tile_off(long long row, int k, int Kpad) {
  const int KS = a_slice_width(Kpad);
  return static_cast<size_t>(row / kRows) * kRows * Kpad + static_cast<size_t>(k / KS) * kRows * KS +
         canon_off(static_cast<int>(row % kRows), k % KS, KS);
}

uint16_t host_bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return static_cast<uint16_t>(u >> 16);  // inf/nan
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;  // round to nearest even
  return static_cast<uint16_t>(u >> 16);
}
float host_bf16_float(uint16_t b) {
  const uint32_t u = static_cast<uint32_t>(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// ---------------------------------------------------------------------------
// Step 2 + operand packing: DFT over q of Zhat[pair][q][zeta] (forward sign,
// eq. fbk3 Step 2), then (Re Z, Im Z) split into bf16 hi/lo in the core-matrix
// layout of the Step-3 A operand. One block per (pair, 8 zetas); the blocks of
// one pair are adjacent in the grid so that they share the pair's cache lines.
// ---------------------------------------------------------------------------
// L = 2Q as a compile-time constant for the common lengths (0 = run-time length).
template <int LC>
__global__ void __launch_bounds__(256) k_fft_pack(const float2* __restrict__ zhat, int Hh, int two_Q_rt, int Kpad,
                                                  FftSchedule sch, const float2* __restrict__ tw_g,
                                                  uint16_t* __restrict__ zhi, uint16_t* __restrict__ zlo,
                                                  int x3) {
  extern __shared__ float2 sh[];
  const int two_Q = LC ? LC : two_Q_rt;
  const int PS = LC ? LC + 4 : two_Q_rt;  // padded row stride of the 8 transforms
  float2* tw = sh;
  float2* b0 = sh + two_Q;
  float2* b1 = b0 + 8 * PS;
  const int ngroups = Kpad / 16;
  const int pair = blockIdx.x / ngroups;
  const int g = blockIdx.x - pair * ngroups;
  for (int e = threadIdx.x; e < two_Q; e += blockDim.x) tw[e] = tw_g[e];
  // Zhat layout [pair][q][zeta] (zeta stride Hs = Hh rounded up to even): 8
  // consecutive zetas per q are one 64-byte segment
  const int Hs = (Hh + 1) & ~1;
  const float2* src = zhat + static_cast<size_t>(pair) * Hs * two_Q;
  for (int e = threadIdx.x; e < 8 * two_Q; e += blockDim.x) {
    const int zl = e & 7, q = e >> 3;
    const int z = g * 8 + zl;
    b0[zl * PS + q] = z < Hh ? src[static_cast<size_t>(q) * Hs + z] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* res;
  if constexpr (LC != 0) res = stockham_fft_c<LC, LC + 4>(b0, b1, 8, tw);
  else res = stockham_fft(b0, b1, 8, two_Q, sch.radix, sch.n, tw);
  for (int e = threadIdx.x; e < 2 * two_Q; e += blockDim.x) {
    const int r = e >> 1, h = e & 1;
    const int kg = 2 * g + h;
    float f[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 c = res[(h * 4 + u) * PS + r];
      f[2 * u] = c.x;
      f[2 * u + 1] = c.y;
    }
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      tc::pack2(f[2 * u], f[2 * u + 1], x3, hi[u], lo[u]);
    }
    const long long row = static_cast<long long>(pair) * two_Q + r;
    const size_t off = a_tile_off(row, kg * 8, Kpad);
    *reinterpret_cast<uint4*>(zhi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    if (x3 == tc::kModeBf16x3) *reinterpret_cast<uint4*>(zlo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

// Same operation for L = 32 c: one warp per transform, the DFT in registers and
// lane shuffles (warp_fft); shared memory only stages the coalesced load and the
// transposed store.
// `lin` = 2Q values of q per transform in Zhat; L >= lin rotations out: for L > lin the
// transform is zero-padded (q = 0..Q-1 at t = q, q = -Q..-1 at t = L + q, zeros between),
// which evaluates Step 2 on the finer grid gamma_r = 2 pi r / L (Section 3.2).
template <int L>
__global__ void __launch_bounds__(256) k_fft_pack_w(const float2* __restrict__ zhat, int Hh, int lin, int Kpad,
                                                    const float2* __restrict__ tw_g, uint16_t* __restrict__ zhi,
                                                    uint16_t* __restrict__ zlo, int x3) {
  constexpr int c = L / 32;
  constexpr int PS = L + 4;
  extern __shared__ float2 sh[];
  float2* tw = sh;
  float2* buf = sh + L;  // [8][PS]
  const int ngroups = Kpad / 16;
  const int pair = blockIdx.x / ngroups;
  const int g = blockIdx.x - pair * ngroups;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < L; e += blockDim.x) tw[e] = tw_g[e];
  const int Hs = (Hh + 1) & ~1;
  const float2* src = zhat + static_cast<size_t>(pair) * Hs * lin;
  const int half = lin >> 1;
  for (int e = threadIdx.x; e < 8 * L; e += blockDim.x) {
    const int zl = e & 7, t = e >> 3;
    const int z = g * 8 + zl;
    const int q = t < half ? t : (t >= L - half ? t - L + lin : -1);
    buf[zl * PS + t] = (z < Hh && q >= 0) ? src[static_cast<size_t>(q) * Hs + z] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 v[c];
#pragma unroll
  for (int k = 0; k < c; ++k) v[k] = buf[warp * PS + lane + 32 * k];
  warp_fft<L>(v, tw);
  __syncwarp();
  const int br = __brev(lane) >> 27;
#pragma unroll
  for (int f2 = 0; f2 < c; ++f2) buf[warp * PS + f2 + c * br] = v[f2];
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * L; e += blockDim.x) {
    const int r = e >> 1, h = e & 1;
    const int kg = 2 * g + h;
    float f[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 cv = buf[(h * 4 + u) * PS + r];
      f[2 * u] = cv.x;
      f[2 * u + 1] = cv.y;
    }
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      tc::pack2(f[2 * u], f[2 * u + 1], x3, hi[u], lo[u]);
    }
    const long long row = static_cast<long long>(pair) * L + r;
    const size_t off = a_tile_off(row, kg * 8, Kpad);
    *reinterpret_cast<uint4*>(zhi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    if (x3 == tc::kModeBf16x3) *reinterpret_cast<uint4*>(zlo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

// Same operation with G lanes per transform (G = 8 or 16, c = L / G values per lane):
// fewer shuffle stages than one warp per transform. A block of 128 threads takes
// ZB = 128 / G zetas of one pair per work item and loops over work items, so the
// twiddle table is loaded once per block. Shared-memory row stride PS = 1 mod 16
// (8-byte banks): the coalesced load (consecutive zetas) writes without conflicts;
// results are stored at rho + rho / c (one pad per c values) so that the bit-reversed
// write of a lane group spreads over the banks.
template <int L, int G>
__global__ void __launch_bounds__(128) k_fft_pack_g(const float2* __restrict__ zhat, int Hh, int lin, int Kpad,
                                                    long long n_items, const float2* __restrict__ tw_g,
                                                    uint16_t* __restrict__ zhi, uint16_t* __restrict__ zlo,
                                                    int x3) {
  constexpr int c = L / G;
  constexpr int ZB = 128 / G;
  constexpr int PS = ((L + G + 15) / 16) * 16 + 1;
  extern __shared__ float2 sh[];
  float2* tw = sh;
  float2* buf = sh + L;  // [ZB][PS]
  for (int e = threadIdx.x; e < L; e += blockDim.x) tw[e] = tw_g[e];
  const int Hs = (Hh + 1) & ~1;
  const int half = lin >> 1;
  const int zchunks = (Kpad / 2 + ZB - 1) / ZB;
  const int tid = threadIdx.x;
  const int grp = tid / G;  // transform (zeta) of this lane within the block
  const int br = __brev(tid & (G - 1)) >> (32 - __ffs(G) + 1);
  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const long long pair = item / zchunks;
    const int z0 = static_cast<int>(item - pair * zchunks) * ZB;
    const float2* src = zhat + static_cast<size_t>(pair) * Hs * lin;
    __syncthreads();  // the previous item's reads of buf (and the twiddle fill) are done
    for (int e = tid; e < ZB * L; e += blockDim.x) {
      const int zl = e % ZB, t = e / ZB;
      const int z = z0 + zl;
      const int q = t < half ? t : (t >= L - half ? t - L + lin : -1);
      buf[zl * PS + t] = (z < Hh && q >= 0) ? src[static_cast<size_t>(q) * Hs + z] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 v[c];
#pragma unroll
    for (int k = 0; k < c; ++k) v[k] = buf[grp * PS + (tid & (G - 1)) + G * k];
    __syncthreads();
    group_fft<L, G>(v, tw);
#pragma unroll
    for (int f2 = 0; f2 < c; ++f2) buf[grp * PS + f2 + (c + 1) * br] = v[f2];
    __syncthreads();
    // rows r of the pair x chunks of 4 complex zetas; (r & 7) fastest, then the chunk,
    // then the row group: consecutive threads write consecutive 16-byte pieces
    constexpr int NC = ZB / 4;
    for (int e = tid; e < L * NC; e += blockDim.x) {
      const int r7 = e & 7;
      const int rest = e >> 3;
      const int kc = rest % NC;
      const int r = (rest / NC) * 8 + r7;
      const int pos = r + r / c;
      const int kg = z0 / 4 + kc;
      if (kg * 4 >= Kpad / 2) continue;
      float f[8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 cv = buf[(kc * 4 + u) * PS + pos];
        f[2 * u] = cv.x;
        f[2 * u + 1] = cv.y;
      }
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        tc::pack2(f[2 * u], f[2 * u + 1], x3, hi[u], lo[u]);
      }
      const long long row = pair * L + r;
      const size_t off = a_tile_off(row, kg * 8, Kpad);
      *reinterpret_cast<uint4*>(zhi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      if (x3 == tc::kModeBf16x3) *reinterpret_cast<uint4*>(zlo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

// Step 2 + packing as a two-factor DFT, 2Q = 12 N1 (q = 12 n1 + n2, r = k1 + N1 k2):
// pass A takes a length-N1 DFT over n1 of every (n2, zeta) from registers and applies
// the twiddle w_2Q^{n2 k1}; pass B a length-12 DFT over n2 of every (k1, zeta). A unit is
// one pair and a block of kZB2 zetas (the padded ones, Hh <= zeta < Kpad / 2, come out
// as zeros). In pass B a warp takes 8 k1 x 4 zetas, so each of its stores (hi, then lo)
// is one whole 128-byte core matrix of the Step-3 A operand (8 rows x 8 K elements).
constexpr int kZB2 = 16;
constexpr int kIS2 = (12 * kZB2 / 16) * 16 + 2;  // U row stride, = 2 mod 16 (8-byte words)

// KS: the K-slice width of the Step-3 A operand (a_slice_width(Kpad): 64, 32 or 16), a compile-time
// constant so that the output offsets need no division. In pass B a warp takes 8 k1 x 8 zetas,
// a lane two adjacent zetas: its two outputs per rotation are 4 consecutive K columns, one 8-byte
// store per part, and a store instruction writes two whole 128-byte core matrices.
template <int N1, int KS>
__global__ void __launch_bounds__(256, 2) k_fft_pack_2f(const float2* __restrict__ zhat, int Hh, int Kpad,
                                                        long long n_units, const float2* __restrict__ tw_g,
                                                        uint16_t* __restrict__ zhi, uint16_t* __restrict__ zlo,
                                                        int mode) {
  constexpr int L = 12 * N1;
  extern __shared__ float2 sh2[];
  float2* tw = sh2;         // [L]
  float2* inter = sh2 + L;  // U [k1][kIS2]: (n2, zeta) at n2 kZB2 + zeta
  for (int e = threadIdx.x; e < L; e += blockDim.x) tw[e] = tw_g[e];
  const int Hs = (Hh + 1) & ~1;
  const int nzb = (Kpad / 2 + kZB2 - 1) / kZB2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (long long u = blockIdx.x; u < n_units; u += gridDim.x) {
    const long long pair = u / nzb;
    const int z0 = static_cast<int>(u - pair * nzb) * kZB2;
    // the pair of this block's next unit into L2, by the one block whose next unit is that pair's
    // first zeta block (its other blocks run alongside), so that pass A's strided rows hit L2
    const long long un = u + gridDim.x;
    if (threadIdx.x == 0 && un < n_units && un % nzb == 0)
      tc::prefetch_l2(zhat + static_cast<size_t>(un / nzb) * L * Hs,
                      static_cast<uint32_t>(static_cast<size_t>(L) * Hs * sizeof(float2)));
    __syncthreads();  // the previous unit's pass-B reads (and the twiddle fill) are done
    const float2* src = zhat + static_cast<size_t>(pair) * L * Hs;
    for (int e = tid; e < 12 * kZB2; e += blockDim.x) {
      const int n2 = e / kZB2;
      const int z = z0 + (e - n2 * kZB2);
      float2 x[N1];
      if (z < Hh) {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = __ldg(src + static_cast<size_t>(12 * n1 + n2) * Hs + z);
        dft_reg<N1>(x, tw, L / N1);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) inter[k1 * kIS2 + e] = k1 ? cmul(x[k1], tw[n2 * k1]) : x[k1];
      } else {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) inter[k1 * kIS2 + e] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    constexpr int n_kb = N1 / 8;
    for (int t = warp; t < n_kb * (kZB2 / 8); t += blockDim.x / 32) {
      const int kb = t % n_kb, zo = t / n_kb;
      const int k1 = kb * 8 + (lane & 7);
      const int zl = zo * 8 + 2 * (lane >> 3);  // this lane's zetas: zl and zl + 1
      const int z = z0 + zl;
      if (2 * z >= Kpad) continue;  // Kpad is a multiple of 16 and z even: 2z + 3 < Kpad too
      float2 va[12], vb[12];
#pragma unroll
      for (int n2 = 0; n2 < 12; ++n2) {
        const float4 w = *reinterpret_cast<const float4*>(inter + k1 * kIS2 + n2 * kZB2 + zl);
        va[n2] = make_float2(w.x, w.y);
        vb[n2] = make_float2(w.z, w.w);
      }
      dft_reg<12>(va, tw, L / 12);
      dft_reg<12>(vb, tw, L / 12);
      // element offset of (row, k = 2z) in the A layout [tile][slice][128 rows][KS]: the K part
      // is the same for every row of this lane
      const int k = 2 * z;
      const size_t kpart = static_cast<size_t>(k / KS) * kRows * KS + ((k % KS) >> 3) * 64 + (k & 7);
      const long long row0 = pair * L + k1;
#pragma unroll
      for (int k2 = 0; k2 < 12; ++k2) {
        const long long row = row0 + N1 * k2;
        const int r = static_cast<int>(row & (kRows - 1));
        const size_t off = static_cast<size_t>(row / kRows) * kRows * Kpad + kpart + (r >> 3) * 8 * KS + (r & 7) * 8;
        uint32_t ha, la, hb, lb;
        tc::pack2(va[k2].x, va[k2].y, mode, ha, la);
        tc::pack2(vb[k2].x, vb[k2].y, mode, hb, lb);
        *reinterpret_cast<uint2*>(zhi + off) = make_uint2(ha, hb);
        if (mode == tc::kModeBf16x3) *reinterpret_cast<uint2*>(zlo + off) = make_uint2(la, lb);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Step 3 (tcgen05) + epilogue. Warp roles: 0 = bulk-copy producer (and TMEM
// allocator), 1 = MMA issuer, 2..9 = epilogue (two sets of four warps, one TMEM
// lane quadrant per warp).
// ---------------------------------------------------------------------------
struct Step3Args {
  const uint16_t* zhi;
  const uint16_t* zlo;
  const uint16_t* yhi;
  const uint16_t* ylo;
  int Kpad, n_tiles, R, G, n_groups, N, two_Q;
  int nj, i0, j0, NT;
  float* scores;
  unsigned long long* keys;
  int* err;
  int x3, nsa;
  // per-image template lists [NI][nj] (NULL: templates j0 + jl) and shift windows
  // (NULL: every shift): shift s counts for image i if max(|s - center_i|) <= window
  const int* list;
  const float2* shifts;
  const float2* center;
  float window;
  // the template part of a key's pose index: j - jbase, or the list position jl (key_pos)
  int jbase, key_pos;
};

__device__ __forceinline__ unsigned int order_key(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Maximum of v[0..W-1] (W = 16, 32 or 64): four independent chains.
template <int W>
__device__ __forceinline__ float max_of(const float* v) {
  float t0 = fmaxf(v[0], v[1]), t1 = fmaxf(v[2], v[3]), t2 = fmaxf(v[4], v[5]), t3 = fmaxf(v[6], v[7]);
#pragma unroll
  for (int x = 8; x < W; x += 8) {
    t0 = fmaxf(t0, fmaxf(v[x], v[x + 1]));
    t1 = fmaxf(t1, fmaxf(v[x + 2], v[x + 3]));
    t2 = fmaxf(t2, fmaxf(v[x + 4], v[x + 5]));
    t3 = fmaxf(t3, fmaxf(v[x + 6], v[x + 7]));
  }
  return fmaxf(fmaxf(t0, t1), fmaxf(t2, t3));
}

// One chunk of W accumulator columns of one row, ns <= W of them valid shifts (the first
// is shift s0): stores the scores (out: the row's score at shift s0, consecutive shifts
// 2Q apart; NULL: no scores) and folds the chunk into the row's running maximum best_v.
// The chunk's argmax is searched only where the maximum reaches thr, the order key of the
// image's best pose so far (a row below it cannot take the image's pose): best_s is then
// the shift of best_v whenever order_key(best_v) >= thr. Ties keep the lowest shift, as
// the keys' pose order does.
template <int W>
__device__ __forceinline__ void step3_chunk(const Step3Args& a, const float* v, int ns, int s0, float* out,
                                            float2 cen, uint32_t thr, float& best_v, int& best_s) {
  if (out) {
#pragma unroll
    for (int x = 0; x < W; ++x)
      if (x < ns) out[static_cast<size_t>(x) * a.two_Q] = v[x];
  }
  if (!a.keys) return;
  if (a.center) {
    float m = -INFINITY;
    int xs = 0;
#pragma unroll
    for (int x = 0; x < W; ++x) {
      if (x < ns) {
        const float2 sh = __ldg(a.shifts + s0 + x);
        if (fabsf(sh.x - cen.x) <= a.window && fabsf(sh.y - cen.y) <= a.window && v[x] > m) {
          m = v[x];
          xs = x;
        }
      }
    }
    if (m > best_v) {
      best_v = m;
      best_s = s0 + xs;
    }
    return;
  }
  float m;
  if (ns == W) {
    m = max_of<W>(v);
  } else {
    m = -INFINITY;
#pragma unroll
    for (int x = 0; x < W; ++x)
      if (x < ns) m = fmaxf(m, v[x]);
  }
  if (m > best_v) {
    best_v = m;
    if (order_key(m) >= thr) {
      int xs = 0;
#pragma unroll
      for (int x = W - 1; x >= 0; --x)
        if (x < ns && v[x] == m) xs = x;
      best_s = s0 + xs;
    }
  }
}

constexpr int kStep3EpiThreads = 128;  // one set of four epilogue warps arrives per tile

__global__ void __launch_bounds__(320, 1) k_step3_tc(const Step3Args a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int parts = tc::mode_split(a.x3) ? 2 : 1;
  const int KS = a_slice_width(a.Kpad);
  const int n_slices = a.Kpad / KS;
  const uint32_t a_part = kRows * KS * 2;    // bytes of one K-slice of one A part (hi or lo)
  const uint32_t y_part = a.G * a.Kpad * 2;  // bytes of one B part
  uint8_t* Ys = smem;
  uint8_t* A0 = smem + static_cast<size_t>(parts) * y_part;
  uint64_t* bars = reinterpret_cast<uint64_t*>(A0 + static_cast<size_t>(a.nsa) * parts * a_part);
  uint64_t* y_full = bars;
  uint64_t* a_full = y_full + 1;
  uint64_t* a_empty = a_full + a.nsa;
  uint64_t* d_full = a_empty + a.nsa;
  uint64_t* d_empty = d_full + 2;
  uint64_t* done_bar = d_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int group = blockIdx.x % a.n_groups;
  const int cta_in_group = blockIdx.x / a.n_groups;
  const int ctas_per_group = gridDim.x / a.n_groups;
  const uint32_t stage_bytes = a_part * parts;

  if (threadIdx.x == 0) {
    tc::mbar_init(y_full, 1);
    for (int s = 0; s < a.nsa; ++s) {
      tc::mbar_init(&a_full[s], 1);
      tc::mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&d_full[s], 1);
      tc::mbar_init(&d_empty[s], kStep3EpiThreads);
    }
    tc::mbar_init(done_bar, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc<kTmemCols>(tmem_slot);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer ----------------
      const size_t goff = static_cast<size_t>(group) * a.G * a.Kpad;
      tc::mbar_arrive_expect_tx(y_full, y_part * parts);
      tc::bulk_g2s(Ys, a.yhi + goff, y_part, y_full);
      if (tc::mode_split(a.x3)) tc::bulk_g2s(Ys + y_part, a.ylo + goff, y_part, y_full);
      int ua = 0;
      bool ok = true;
      for (int t = cta_in_group; t < a.n_tiles && ok; t += ctas_per_group) {
        for (int sl = 0; sl < n_slices; ++sl) {
          const int sa = ua % a.nsa;
          if (!(ok = tc::mbar_wait(&a_empty[sa], ((ua / a.nsa) & 1) ^ 1, abort_flag, a.err))) break;
          tc::mbar_arrive_expect_tx(&a_full[sa], stage_bytes);
          uint8_t* dst = A0 + static_cast<size_t>(sa) * parts * a_part;
          const size_t toff = static_cast<size_t>(t) * kRows * a.Kpad + static_cast<size_t>(sl) * kRows * KS;
          tc::bulk_g2s(dst, a.zhi + toff, a_part, &a_full[sa]);
          if (tc::mode_split(a.x3)) tc::bulk_g2s(dst + a_part, a.zlo + toff, a_part, &a_full[sa]);
          ++ua;
        }
      }
      // drain copies that may still be in flight before the CTA exits
      volatile int never = 0;
      tc::mbar_wait(y_full, 0, &never, a.err, 100000000ull);
      if (!ok)
        for (int u = ua - a.nsa; u < ua; ++u)
          if (u >= 0) tc::mbar_wait(&a_full[u % a.nsa], (u / a.nsa) & 1, &never, a.err, 100000000ull);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (the whole warp; one elected lane issues) ----------------
    // The issue loop is on the critical path of the tensor pipe: stage index and phase are
    // kept as counters, and the K steps of a 32- or 64-wide slice are issued unrolled.
    const unsigned FULL = 0xFFFFFFFFu;
    const uint32_t idesc = tc::idesc_f32acc(kRows, a.G, a.x3);
    const uint32_t sbo_y = a.Kpad * 16;  // 8-row group stride of B (full K per group)
    const uint32_t sbo_a = KS * 16;      // 8-row group stride of an A slice
    // descriptors are advanced by adding (byte offset >> 4) to the start-address field
    const uint64_t dy0 = tc::smem_desc(tc::smem_u32(Ys), 128, sbo_y);
    const uint64_t da0 = tc::smem_desc(tc::smem_u32(A0), 128, sbo_a);
    const uint64_t y_lo_step = y_part >> 4, a_lo_step = a_part >> 4;
    const uint64_t a_stage_step = (static_cast<uint64_t>(parts) * a_part) >> 4;
    const bool split = tc::mode_split(a.x3);
    int sa = 0, ud = 0;
    uint32_t ph = 0;
    bool ok = __all_sync(FULL, tc::mbar_wait(y_full, 0, abort_flag, a.err));
    tc::tc_fence_after();
    for (int t = cta_in_group; t < a.n_tiles && ok; t += ctas_per_group) {
      const int sd = ud & 1;
      if (!(ok = __all_sync(FULL, tc::mbar_wait(&d_empty[sd], ((ud >> 1) & 1) ^ 1, abort_flag, a.err)))) break;
      tc::tc_fence_after();
      const uint32_t d_tmem = tmem_base + sd * a.G;
      for (int sl = 0; sl < n_slices; ++sl) {
        if (!(ok = __all_sync(FULL, tc::mbar_wait(&a_full[sa], ph, abort_flag, a.err)))) break;
        tc::tc_fence_after();
        const uint64_t dah = da0 + sa * a_stage_step;
        const uint64_t dbh = dy0 + static_cast<uint64_t>(sl * (KS / 16)) * 16;  // B: two core matrices per k-step
        if (split && KS == 32) {
          tc::mma_bf16x3_ss_warp(d_tmem, dah, dah + a_lo_step, dbh, dbh + y_lo_step, idesc, sl > 0 ? 1u : 0u);
          tc::mma_bf16x3_ss_warp(d_tmem, dah + 16, dah + 16 + a_lo_step, dbh + 16, dbh + 16 + y_lo_step, idesc, 1u);
        } else if (split && KS == 64) {
          tc::mma_bf16x3_ss_warp(d_tmem, dah, dah + a_lo_step, dbh, dbh + y_lo_step, idesc, sl > 0 ? 1u : 0u);
          tc::mma_bf16x3_ss_warp(d_tmem, dah + 16, dah + 16 + a_lo_step, dbh + 16, dbh + 16 + y_lo_step, idesc, 1u);
          tc::mma_bf16x3_ss_warp(d_tmem, dah + 32, dah + 32 + a_lo_step, dbh + 32, dbh + 32 + y_lo_step, idesc, 1u);
          tc::mma_bf16x3_ss_warp(d_tmem, dah + 48, dah + 48 + a_lo_step, dbh + 48, dbh + 48 + y_lo_step, idesc, 1u);
        } else {
          for (int kk = 0; kk < KS / 16; ++kk) {
            const uint32_t acc = (sl > 0 || kk > 0) ? 1u : 0u;
            const uint64_t o = static_cast<uint64_t>(kk) * 16;
            if (split)
              tc::mma_bf16x3_ss_warp(d_tmem, dah + o, dah + o + a_lo_step, dbh + o, dbh + o + y_lo_step, idesc, acc);
            else
              tc::mma_bf16_ss_warp(d_tmem, dah + o, dbh + o, idesc, acc);
          }
        }
        tc::mma_commit_warp(&a_empty[sa]);
        if (++sa == a.nsa) {
          sa = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      tc::mma_commit_warp(&d_full[sd]);
      ++ud;
    }
    // wait for every issued MMA before teardown
    tc::mma_commit_warp(done_bar);
    volatile int never = 0;
    tc::mbar_wait(done_bar, 0, &never, a.err, 200000000ull);
  } else {
    // ---------------- epilogue ----------------
    // Two sets of four warps; set e handles the tiles that land in accumulator e, so that
    // the TMEM loads of one set overlap the arithmetic of the other (warp w reads TMEM lane
    // quadrant w % 4).
    const int eset = (warp - 2) >> 2;
    const int quad = warp & 3;
    const unsigned FULL = 0xFFFFFFFFu;
    const int g0 = group * a.G;  // first shift of this CTA's group
    int ud = 0;
    bool ok = true;
    for (int t = cta_in_group; t < a.n_tiles && ok; t += ctas_per_group, ++ud) {
      if ((ud & 1) != eset) continue;
      const int row = t * kRows + quad * 32 + lane;
      const bool valid = row < a.R;
      const int pair = valid ? row / a.two_Q : 0;
      const int r = valid ? row - pair * a.two_Q : 0;
      const int il = pair / a.nj, jl = pair - il * a.nj;
      const int i = a.i0 + il;
      const int j = a.list ? __ldg(a.list + static_cast<size_t>(i) * a.nj + jl) : a.j0 + jl;
      const float2 cen = (a.keys && a.center && valid) ? a.center[i] : make_float2(0.f, 0.f);
      // the image's best key so far (keys only grow: a stale value prunes less, never wrongly)
      const uint32_t thr =
          (a.keys && !a.center && valid) ? static_cast<uint32_t>(__ldcg(a.keys + i) >> 32) : 0u;
      const int sd = eset;
      bool w = tc::mbar_wait(&d_full[sd], (ud >> 1) & 1, abort_flag, a.err);
      if (!(ok = __all_sync(FULL, w))) break;
      tc::tc_fence_after();
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quad * 32) << 16) + sd * a.G;
      float best_v = -INFINITY;
      int best_s = 0;
      float* out = a.scores ? a.scores + ((static_cast<size_t>(i) * a.NT + j) * a.N + g0) * a.two_Q + r : nullptr;
      for (int c0 = 0; c0 < a.G;) {
        const int cw = a.G - c0 >= 64 ? 64 : (a.G - c0 >= 32 ? 32 : 16);  // G is a multiple of 16
        float v[64];
        if (cw == 64)
          tc::tmem_ld64(taddr + c0, v);
        else if (cw == 32)
          tc::tmem_ld32(taddr + c0, v);
        else
          tc::tmem_ld16(taddr + c0, v);
        if (c0 + cw >= a.G) {  // the accumulator is free once its last columns are in registers
          tc::tc_fence_before();
          tc::mbar_arrive(&d_empty[sd]);
        }
        const int ns = valid ? min(cw, a.N - (g0 + c0)) : 0;
        if (ns > 0) {
          float* o = out ? out + static_cast<size_t>(c0) * a.two_Q : nullptr;
          if (cw == 64)
            step3_chunk<64>(a, v, ns, g0 + c0, o, cen, thr, best_v, best_s);
          else if (cw == 32)
            step3_chunk<32>(a, v, ns, g0 + c0, o, cen, thr, best_v, best_s);
          else
            step3_chunk<16>(a, v, ns, g0 + c0, o, cen, thr, best_v, best_s);
        }
        c0 += cw;
      }
      if (a.keys) {
        unsigned long long key = 0ull;
        if (valid && best_v > -INFINITY && order_key(best_v) >= thr) {
          const unsigned int jk = static_cast<unsigned int>(a.key_pos ? jl : j - a.jbase);
          const unsigned int idx = (jk * a.two_Q + r) * static_cast<unsigned int>(a.N) + best_s;
          key = (static_cast<unsigned long long>(order_key(best_v)) << 32) | (0xFFFFFFFFu - idx);
        }
        const int img = key ? i : -1;
        unsigned pending = __ballot_sync(FULL, key != 0ull);
        while (pending) {
          const int leader = __ffs(pending) - 1;
          const int limg = __shfl_sync(FULL, img, leader);
          const bool mine = key != 0ull && img == limg;
          const unsigned grp = __ballot_sync(FULL, mine);
          unsigned long long kk = mine ? key : 0ull;
#pragma unroll
          for (int off = 16; off; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(FULL, kk, off);
            kk = o > kk ? o : kk;
          }
          if (lane == leader) atomicMax(a.keys + limg, kk);
          pending &= ~grp;
        }
      }
    }
  }

  __syncwarp();  // the single-lane producer rejoins its warp
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc<kTmemCols>(tmem_base);
}

int kpad_of(const ftk_plan_s* p) { return (2 * p->Hh + 15) / 16 * 16; }

constexpr int kMaxAStages = 12;

size_t step3_smem(int Kpad, int G, int parts, int nsa) {
  return static_cast<size_t>(parts) * G * Kpad * 2 + static_cast<size_t>(nsa) * parts * kRows * a_slice_width(Kpad) * 2 +
         (1 + 2 * nsa + 4 + 1) * 8 + 16 + 64;
}

// Smallest number of shift groups (with G <= gmax) whose resident B slice leaves room
// for at least `min_stages` A K-slice stages; uses as many stages as fit (<= 12).
bool choose_groups(int N, int Kpad, int* G, int* n_groups, int* nsa, int gmax = 256, int min_stages = 4) {
  for (int need = min_stages; need >= 1; need = need > 1 ? need / 2 : 0) {
    for (int ng = 1; ng <= 1024; ++ng) {
      const int g = ((N + ng - 1) / ng + 15) / 16 * 16;
      if (g > gmax) continue;
      if (step3_smem(Kpad, g, 2, need) <= kSmemBudget) {
        int st = need;
        while (st < kMaxAStages && step3_smem(Kpad, g, 2, st + 1) <= kSmemBudget) ++st;
        *G = g;
        *n_groups = ng;
        *nsa = st;
        return true;
      }
    }
    if (need == 1) break;
  }
  return false;
}

}  // namespace

bool tc_supported(const ftk_plan_s* p) {
  int G, ng, nsa;
  return p->two_Q % 8 == 0 && choose_groups(p->N, kpad_of(p), &G, &ng, &nsa) && step1_tc_supported(p);
}

namespace {

constexpr size_t kAl = 256;
size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

// Scratch of one chunk of ib images x tb templates (bytes), excluding the keys, with the
// packed Step-1 operands of tpack templates (tb, or all templates packed once).
size_t tc_chunk_bytes(const ftk_plan_s* p, long long ib, long long tb, long long tpack) {
  const long long tb_pad = (tpack + kRows - 1) / kRows * kRows;
  const long long rows = ib * tb * p->n_rot;
  const long long tiles = (rows + kRows - 1) / kRows;
  return al(static_cast<size_t>(tb_pad) * step1_template_row_bytes(p)) + al(static_cast<size_t>(ib) * step1_image_bytes(p)) +
         al(static_cast<size_t>(ib) * tb * ((p->Hh + 1) & ~1) * p->two_Q * sizeof(float2)) +
         al(static_cast<size_t>(tiles) * kRows * kpad_of(p) * 2 * 2);
}

// Step 1 runs its (image, 128-template tile) work units round-robin over the SMs, one unit
// per SM at a time (a block with fewer units than SMs is split along q, as step1_tc_launch
// does). The fraction of SM-rounds that chunking NI x NT pairs into blocks of ib images x tb
// templates keeps busy, over the whole search.
double chunk_efficiency(long long NI, long long NT, long long ib, long long tb, int nsm, int two_Q) {
  double work = 0, time = 0;
  auto add = [&](long long ni, long long nj, long long count) {
    if (count <= 0 || ni <= 0 || nj <= 0) return;
    const long long u = ni * ((nj + kRows - 1) / kRows);
    const long long qs = u < nsm ? std::min<long long>(two_Q, (nsm + u - 1) / u) : 1;
    work += static_cast<double>(u) * count;
    time += static_cast<double>((u * qs + nsm - 1) / nsm) / qs * count;
  };
  const long long fi = NI / ib, ri = NI % ib, ft = NT / tb, rt = NT % tb;
  add(ib, tb, fi * ft);
  add(ri, tb, ft);
  add(ib, rt, fi);
  add(ri, rt, 1);
  return time > 0 ? work / (time * nsm) : 1.0;
}

// Chunk shape (ib images x tb templates) of a search of NI x NT pairs within `limit` bytes
// of scratch. Template blocks hold at most 4096 templates (where `wide`, fewer than 2^32 pose
// indices); among template blocks of that size or half of it and the image counts that fit,
// the shape whose Step-1 rounds leave the fewest SMs idle, then the one with the most pairs
// per chunk. Where all NT templates' packed operands fit beside the chunk (*tpack_out = NT),
// they are packed once and the images of a chunk once for all template blocks; else each
// template block is packed in turn (*tpack_out = tb). At n = 128 with 8192 x 4096 pairs and
// 16 GiB that is 19 images x 2048 templates: 304 units, two full rounds of 152 SMs.
ftk_status choose_chunk(const ftk_plan_s* p, int NI, int NT, size_t limit, bool wide, long long* ib_out,
                        long long* tb_out, long long* tpack_out) {
  long long tb0 = std::max(1, std::min(NT, 4096));
  while (wide && tb0 > 1 && pose_index_wide(tb0, p->n_rot, p->N)) tb0 /= 2;
  if (wide && pose_index_wide(tb0, p->n_rot, p->N)) return FTK_ERR_UNSUPPORTED;
  while (tb0 > 1 && tc_chunk_bytes(p, 1, tb0, tb0) > limit)
    tb0 = tb0 > kRows ? (tb0 / 2 + kRows - 1) / kRows * kRows : tb0 / 2;
  if (tc_chunk_bytes(p, 1, tb0, tb0) > limit) return FTK_ERR_NOMEM;
  int nsm = 148;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || nsm < 1) nsm = 148;
  const long long cap = std::min<long long>(std::max(NI, 1), 65535);
  double best_e = -1.0;
  long long best_ib = 1, best_tb = tb0, best_tpack = tb0;
  for (long long tb = tb0;;) {
    // the shared pack of all templates where it fits beside a one-image chunk (tb is then a
    // multiple of 128, so the blocks start on template tiles)
    const long long tpack = (NT > tb && tb % kRows == 0 && tc_chunk_bytes(p, 1, tb, NT) <= limit) ? NT : tb;
    if (tc_chunk_bytes(p, 1, tb, tpack) <= limit) {
      long long lo = 1, hi = cap;  // the largest image block that fits: bytes grow with ib
      while (lo < hi) {
        const long long mid = (lo + hi + 1) / 2;
        if (tc_chunk_bytes(p, mid, tb, tpack) <= limit) lo = mid;
        else hi = mid - 1;
      }
      for (long long ib = lo; ib >= std::max(1LL, lo / 2); --ib) {
        const double e = chunk_efficiency(NI, NT, ib, tb, nsm, p->two_Q);
        if (e > best_e + 1e-3 || (e > best_e - 1e-3 && ib * tb > best_ib * best_tb)) {
          if (e > best_e) best_e = e;
          best_ib = ib;
          best_tb = tb;
          best_tpack = tpack;
        }
      }
    }
    if (tb <= kRows || 2 * tb < tb0) break;  // candidates: tb0 and tb0 / 2 (multiples of 128)
    tb = (tb / 2 + kRows - 1) / kRows * kRows;
  }
  *ib_out = best_ib;
  *tb_out = best_tb;
  *tpack_out = best_tpack;
  return FTK_OK;
}

}  // namespace

void tc_workspace(const ftk_plan_s* p, int NI, int NT, size_t* min_bytes, size_t* good_bytes) {
  const long long tb_min = std::max(1, std::min(NT, kRows));
  if (min_bytes) *min_bytes = tc_chunk_bytes(p, 1, tb_min, tb_min);
  if (good_bytes) {
    long long ib = 1, tb = std::max(1, std::min(NT, 4096)), tpack = tb;
    if (choose_chunk(p, NI, NT, size_t(1) << 34, false, &ib, &tb, &tpack) != FTK_OK) {  // <= 16 GiB
      ib = 1;
      tb = tpack = tb_min;
    }
    *good_bytes = tc_chunk_bytes(p, ib, tb, tpack);
  }
}

namespace {

__global__ void k_to_f16(const float* __restrict__ src, long long n, __half* __restrict__ dst) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x)
    dst[e] = __float2half_rn(src[e]);
}

// Uploads FP32 values and rounds them to FP16 on the device into a new buffer.
cudaError_t upload_f16(const std::vector<float>& v, uint16_t** out) {
  float* tmp = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&tmp), v.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(out), v.size() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMemcpy(tmp, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const long long n = static_cast<long long>(v.size());
    k_to_f16<<<static_cast<unsigned>(std::min<long long>((n + 255) / 256, 4096)), 256>>>(tmp, n,
                                                                                         reinterpret_cast<__half*>(*out));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(tmp);
  return e;
}

}  // namespace

cudaError_t tc_build_tables(ftk_plan_s* p, const std::vector<float2>& Y) {
  const int Kpad = kpad_of(p);
  p->tc.Kpad = Kpad;
  for (int& m : p->tc.max_clusters) m = -1;
  const int gmax = p->tune.step3_group_max > 0 ? p->tune.step3_group_max : 256;
  // default: at least 64 KB of A stages in flight (two 64-wide slices, four 32-wide)
  const int stages = p->tune.step3_a_stages > 0 ? p->tune.step3_a_stages : (a_slice_width(Kpad) == 64 ? 2 : 4);
  if (!choose_groups(p->N, Kpad, &p->tc.G, &p->tc.n_groups, &p->tc.nsa, gmax, stages)) return cudaSuccess;
  const int rows = p->tc.G * p->tc.n_groups;
  std::vector<uint16_t> hi(static_cast<size_t>(rows) * Kpad, 0), lo(static_cast<size_t>(rows) * Kpad, 0);
  for (int s = 0; s < p->N; ++s) {
    for (int z = 0; z < p->Hh; ++z) {
      const float2 y = Y[static_cast<size_t>(s) * p->Hh + z];
      const float vals[2] = {y.x, -y.y};
      for (int part = 0; part < 2; ++part) {
        const size_t off = canon_off(s, 2 * z + part, Kpad);
        const uint16_t h = host_bf16_bits(vals[part]);
        hi[off] = h;
        lo[off] = host_bf16_bits(vals[part] - host_bf16_float(h));
      }
    }
  }
  // row-major copy for the fused Steps 2-3 (shift s = TMEM lane, rows padded to 128)
  p->tc.n_mt = (p->N + kRows - 1) / kRows;
  const size_t rrows = static_cast<size_t>(p->tc.n_mt) * kRows;
  std::vector<uint16_t> rhi(rrows * Kpad, 0), rlo(rrows * Kpad, 0);
  for (int s = 0; s < p->N; ++s)
    for (int k = 0; k < Kpad; ++k) {
      const size_t off = canon_off(s, k, Kpad);
      rhi[static_cast<size_t>(s) * Kpad + k] = hi[off];
      rlo[static_cast<size_t>(s) * Kpad + k] = lo[off];
    }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p->tc.d_Yhi), hi.size() * 2);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->tc.d_Ylo), lo.size() * 2);
  if (e == cudaSuccess) e = cudaMemcpy(p->tc.d_Yhi, hi.data(), hi.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->tc.d_Ylo, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->tc.d_Yrhi), rhi.size() * 2);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->tc.d_Yrlo), rlo.size() * 2);
  if (e == cudaSuccess) e = cudaMemcpy(p->tc.d_Yrhi, rhi.data(), rhi.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->tc.d_Yrlo, rlo.data(), rlo.size() * 2, cudaMemcpyHostToDevice);
  // FP16 copies of both layouts: FP32 values in place of the bf16 hi parts, rounded on the device
  if (e == cudaSuccess) {
    std::vector<float> f(static_cast<size_t>(rows) * Kpad, 0.f), fr(rrows * Kpad, 0.f);
    for (int s = 0; s < p->N; ++s)
      for (int z = 0; z < p->Hh; ++z) {
        const float2 y = Y[static_cast<size_t>(s) * p->Hh + z];
        const float vals[2] = {y.x, -y.y};
        for (int part = 0; part < 2; ++part) {
          f[canon_off(s, 2 * z + part, Kpad)] = vals[part];
          fr[static_cast<size_t>(s) * Kpad + 2 * z + part] = vals[part];
        }
      }
    e = upload_f16(f, &p->tc.d_Yh16);
    if (e == cudaSuccess) e = upload_f16(fr, &p->tc.d_Yr16);
  }
  return e;
}

void tc_free_tables(ftk_plan_s* p) {
  cudaFree(p->tc.d_Yh16);
  cudaFree(p->tc.d_Yr16);
  p->tc.d_Yh16 = p->tc.d_Yr16 = nullptr;
  cudaFree(p->tc.d_Yhi);
  cudaFree(p->tc.d_Ylo);
  cudaFree(p->tc.d_Yrhi);
  cudaFree(p->tc.d_Yrlo);
  p->tc.d_Yhi = p->tc.d_Ylo = nullptr;
  p->tc.d_Yrhi = p->tc.d_Yrlo = nullptr;
}

namespace {

template <int LC>
ftk_status launch_fft_pack_t(ftk_plan_s* p, const float2* zbuf, long long blocks, int Kpad, uint16_t* zhi,
                             uint16_t* zlo, int x3, cudaStream_t s) {
  if (p->n_rot != p->two_Q) return FTK_ERR_UNSUPPORTED;  // zero-padding: the warp kernels only
  const int L = p->two_Q;
  const int PS = LC ? LC + 4 : L;
  const size_t smem = (static_cast<size_t>(L) + 16 * PS) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_fft_pack<LC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return FTK_ERR_CUDA;
  FTK_LAUNCH(p, kKFftPack, s,
             (k_fft_pack<LC><<<static_cast<unsigned>(blocks), 256, smem, s>>>(zbuf, p->Hh, L, Kpad, p->fft, p->d_tw,
                                                                               zhi, zlo, x3),
              cudaGetLastError()));
  return FTK_OK;
}

template <int L>
ftk_status launch_fft_pack_w(ftk_plan_s* p, const float2* zbuf, long long blocks, int Kpad, uint16_t* zhi,
                             uint16_t* zlo, int x3, cudaStream_t s) {
  const size_t smem = (static_cast<size_t>(L) + 8 * (L + 4)) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_fft_pack_w<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return FTK_ERR_CUDA;
  const float2* tw = p->n_rot == p->two_Q ? p->d_tw : p->d_tw_rot;
  FTK_LAUNCH(p, kKFftPack, s,
             (k_fft_pack_w<L><<<static_cast<unsigned>(blocks), 256, smem, s>>>(zbuf, p->Hh, p->two_Q, Kpad, tw, zhi,
                                                                                zlo, x3),
              cudaGetLastError()));
  return FTK_OK;
}

template <int L, int G>
ftk_status launch_fft_pack_g(ftk_plan_s* p, const float2* zbuf, long long pairs, int Kpad, uint16_t* zhi,
                             uint16_t* zlo, int x3, cudaStream_t s) {
  constexpr int ZB = 128 / G;
  constexpr int PS = ((L + G + 15) / 16) * 16 + 1;
  const size_t smem = (static_cast<size_t>(L) + static_cast<size_t>(ZB) * PS) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_fft_pack_g<L, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return FTK_ERR_CUDA;
  const long long items = pairs * ((Kpad / 2 + ZB - 1) / ZB);
  const long long grid = std::min<long long>(items, 152LL * 24);
  const float2* tw = p->n_rot == p->two_Q ? p->d_tw : p->d_tw_rot;
  FTK_LAUNCH(p, kKFftPack, s,
             (k_fft_pack_g<L, G><<<static_cast<unsigned>(grid), 128, smem, s>>>(zbuf, p->Hh, p->two_Q, Kpad, items, tw,
                                                                                zhi, zlo, x3),
              cudaGetLastError()));
  return FTK_OK;
}

template <int N1, int KS>
ftk_status launch_fft_pack_2f_ks(ftk_plan_s* p, const float2* zbuf, long long pairs, int Kpad, uint16_t* zhi,
                                 uint16_t* zlo, int x3, cudaStream_t s) {
  const size_t smem = (static_cast<size_t>(12 * N1) + static_cast<size_t>(N1) * kIS2) * sizeof(float2);
  cudaError_t e =
      cudaFuncSetAttribute(k_fft_pack_2f<N1, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return FTK_ERR_CUDA;
  const long long units = pairs * ((Kpad / 2 + kZB2 - 1) / kZB2);
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long grid = std::min<long long>(units, 2LL * nsm);
  FTK_LAUNCH(p, kKFftPack, s,
             (k_fft_pack_2f<N1, KS><<<static_cast<unsigned>(grid), 256, smem, s>>>(zbuf, p->Hh, Kpad, units, p->d_tw,
                                                                                     zhi, zlo, x3),
              cudaGetLastError()));
  return FTK_OK;
}

template <int N1>
ftk_status launch_fft_pack_2f(ftk_plan_s* p, const float2* zbuf, long long pairs, int Kpad, uint16_t* zhi,
                              uint16_t* zlo, int x3, cudaStream_t s) {
  return a_slice_width(Kpad) == 64 ? launch_fft_pack_2f_ks<N1, 64>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s)
         : a_slice_width(Kpad) == 32 ? launch_fft_pack_2f_ks<N1, 32>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s)
                                   : launch_fft_pack_2f_ks<N1, 16>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
}

ftk_status launch_fft_pack(ftk_plan_s* p, const float2* zbuf, long long blocks, int Kpad, uint16_t* zhi, uint16_t* zlo,
                           int x3, cudaStream_t s) {
  const long long pairs = blocks / (Kpad / 16);
  const int lanes = p->tune.fft_lanes;
  if (lanes == 0 && p->n_rot == p->two_Q) {  // the two-factor DFT where 2Q = 12 N1
    switch (p->two_Q) {
      case 96: return launch_fft_pack_2f<8>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      case 192: return launch_fft_pack_2f<16>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      case 288: return launch_fft_pack_2f<24>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      case 384: return launch_fft_pack_2f<32>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      default: break;
    }
  }
  if (lanes == 8) {
    switch (p->n_rot) {
      case 96: return launch_fft_pack_g<96, 8>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      case 192: return launch_fft_pack_g<192, 8>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      default: break;
    }
  } else if (lanes == 0 || lanes == 16) {
    switch (p->n_rot) {
      case 96: return launch_fft_pack_g<96, 16>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      case 192: return launch_fft_pack_g<192, 16>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      case 288: return launch_fft_pack_g<288, 16>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      case 384: return launch_fft_pack_g<384, 16>(p, zbuf, pairs, Kpad, zhi, zlo, x3, s);
      default: break;
    }
  }
  switch (p->n_rot) {
    case 96: return launch_fft_pack_w<96>(p, zbuf, blocks, Kpad, zhi, zlo, x3, s);
    case 192: return launch_fft_pack_w<192>(p, zbuf, blocks, Kpad, zhi, zlo, x3, s);
    case 288: return launch_fft_pack_w<288>(p, zbuf, blocks, Kpad, zhi, zlo, x3, s);
    case 384: return launch_fft_pack_w<384>(p, zbuf, blocks, Kpad, zhi, zlo, x3, s);
    case 576: return launch_fft_pack_w<576>(p, zbuf, blocks, Kpad, zhi, zlo, x3, s);
    case 768: return launch_fft_pack_w<768>(p, zbuf, blocks, Kpad, zhi, zlo, x3, s);
    default: return launch_fft_pack_t<0>(p, zbuf, blocks, Kpad, zhi, zlo, x3, s);
  }
}

Step3Args step3_args(const ftk_plan_s* p, int x3, const uint16_t* zhi, const uint16_t* zlo, int n_tiles, long long R,
                     int nj, int i0, int j0, int NT) {
  Step3Args args;
  args.zhi = zhi;
  args.zlo = zlo;
  args.yhi = x3 == tc::kModeF16 ? p->tc.d_Yh16 : p->tc.d_Yhi;
  args.ylo = p->tc.d_Ylo;
  args.Kpad = p->tc.Kpad;
  args.n_tiles = n_tiles;
  args.R = static_cast<int>(R);
  args.G = p->tc.G;
  args.n_groups = p->tc.n_groups;
  args.N = p->N;
  args.two_Q = p->n_rot;  // rows per pair = rotations
  args.nj = nj;
  args.i0 = i0;
  args.j0 = j0;
  args.NT = NT;
  args.scores = nullptr;
  args.keys = nullptr;
  args.err = p->d_err;
  args.x3 = x3;
  args.nsa = p->tc.nsa;
  args.list = nullptr;
  args.shifts = p->d_shifts;
  args.center = nullptr;
  args.window = 0.f;
  args.jbase = 0;
  args.key_pos = 0;
  return args;
}

ftk_status launch_step3(ftk_plan_s* p, const Step3Args& args, cudaStream_t s) {
  const int parts = tc::mode_split(args.x3) ? 2 : 1;
  // at least half of the SM's shared memory, so that a single CTA (and a single
  // 512-column TMEM allocation) is resident per SM
  const size_t smem = std::max<size_t>(step3_smem(args.Kpad, args.G, parts, args.nsa), 116 * 1024);
  cudaError_t e = cudaFuncSetAttribute(k_step3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return FTK_ERR_CUDA;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_group = std::max(1, std::min(args.n_tiles, nsm / args.n_groups));
  const int grid = per_group * args.n_groups;
  FTK_LAUNCH(p, kKStep3Tc, s, (k_step3_tc<<<grid, 320, smem, s>>>(args), cudaGetLastError()));
  return FTK_OK;
}

// Scratch of one chunk, laid out once for the largest chunk (ib images x tb templates):
// packed templates and images, Zhat, and the Step-3 A operand (hi, lo).
struct ChunkLayout {
  uint16_t* tbuf;
  uint16_t* ibuf;
  float2* zbuf;
  uint16_t* zhi;
  uint16_t* zlo;
};

ChunkLayout chunk_layout(const ftk_plan_s* p, char* work, long long ib, long long tb, long long tpack) {
  ChunkLayout c;
  const long long pairs = ib * tb;
  const int n_tiles = static_cast<int>((pairs * p->n_rot + kRows - 1) / kRows);
  const long long tb_pad = (tpack + kRows - 1) / kRows * kRows;
  c.tbuf = reinterpret_cast<uint16_t*>(work);
  char* w = work + al(static_cast<size_t>(tb_pad) * step1_template_row_bytes(p));
  c.ibuf = reinterpret_cast<uint16_t*>(w);
  w += al(static_cast<size_t>(ib) * step1_image_bytes(p));
  c.zbuf = reinterpret_cast<float2*>(w);
  w += al(static_cast<size_t>(pairs) * ((p->Hh + 1) & ~1) * p->two_Q * sizeof(float2));
  c.zhi = reinterpret_cast<uint16_t*>(w);
  c.zlo = c.zhi + static_cast<size_t>(n_tiles) * kRows * p->tc.Kpad;
  return c;
}

// pack_templates: pack this chunk's templates (b) into L.tbuf first. With a shared pack of all
// templates (shared = true) L.tbuf holds all NT templates' operands and this chunk's start at
// template j0; its images are packed only when pack_images.
ftk_status tc_run_chunk(ftk_plan_s* p, int precision, const float2* a, int ni, const float2* b, int nj, int i0, int j0,
                        int NT, bool pack_templates, const ChunkLayout& L, float* d_scores, unsigned long long* d_keys,
                        const BestRecords& rec, cudaStream_t s, bool shared = false, bool pack_images = true) {
  const int Kpad = p->tc.Kpad;
  const int x3 = op_mode(precision);
  const long long pairs = static_cast<long long>(ni) * nj;
  const long long R = pairs * p->n_rot;
  const int n_tiles = static_cast<int>((R + kRows - 1) / kRows);
  float2* zbuf = L.zbuf;

  // Step 1 (tcgen05) -> Zhat [pair][q][zeta]
  ftk_status st = shared ? step1_tc_run_block(p, precision, a, ni, nj, j0 / kRows, NT, L.tbuf, zbuf, L.ibuf,
                                              pack_images, s)
                         : step1_tc_run(p, precision, a, ni, b, nj, zbuf, L.tbuf, L.ibuf, pack_templates, s);
  if (st != FTK_OK) return st;
  const int jbase = rec.wide ? j0 : 0;  // wide pose indices count from the chunk's first template
  if (!d_scores && d_keys && step23_supported(p, precision))  // Steps 2-3 fused, best pose only
    return step23_run(p, precision, zbuf, pairs, nj, i0, j0, d_keys, nullptr, nullptr, 0.f, jbase, 0, s);
  if (!d_scores && d_keys && step23c_supported(p, precision))  // fused over a cluster (2Q = 128 R)
    return step23c_run(p, precision, zbuf, pairs, nj, i0, j0, d_keys, nullptr, nullptr, 0.f, jbase, 0, s);
  // Step 2 + pack
  {
    const long long blocks = pairs * (Kpad / 16);
    if (blocks > 0x7FFFFFFFLL) return FTK_ERR_UNSUPPORTED;
    st = launch_fft_pack(p, zbuf, blocks, Kpad, L.zhi, L.zlo, x3, s);
    if (st != FTK_OK) return st;
  }
  // Step 3 + epilogue
  Step3Args args = step3_args(p, x3, L.zhi, L.zlo, n_tiles, R, nj, i0, j0, NT);
  args.scores = d_scores;
  args.keys = d_keys;
  args.jbase = jbase;
  return launch_step3(p, args, s);
}

// Steps 1-3 of per-image template lists: chunks of images, Step 1 on the FP32 SIMT
// engine into the tensor-core layout, then the tensor-core Steps 2-3 unchanged.
size_t shortlist_chunk_bytes(const ftk_plan_s* p, long long ni, int K) {
  const long long pairs = ni * K;
  const long long n_tiles = (pairs * p->n_rot + kRows - 1) / kRows;
  size_t bytes = al(static_cast<size_t>(pairs) * ((p->Hh + 1) & ~1) * p->two_Q * sizeof(float2)) +
                 2 * al(static_cast<size_t>(n_tiles) * kRows * p->tc.Kpad * sizeof(uint16_t));
  if (step1_tc_supported(p))
    bytes += al(static_cast<size_t>(ni) * step1_list_template_bytes(p, K)) + al(static_cast<size_t>(ni) * step1_image_bytes(p));
  return bytes;
}

}  // namespace

ftk_status tc_run_all(ftk_plan_s* p, int precision, const float2* a, int NI, const float2* b, int NT, float* d_scores,
                      unsigned long long* d_keys, const BestRecords& rec, char* work, size_t work_bytes,
                      cudaStream_t s) {
  if (!p->tc.d_Yhi) return FTK_ERR_UNSUPPORTED;
  // chunk shape: see choose_chunk (with wide pose indices, template blocks whose indices stay
  // below 2^32)
  long long ib = 1, tb = 1, tpack = 1;
  const ftk_status sc = choose_chunk(p, NI, NT, work_bytes, rec.wide, &ib, &tb, &tpack);
  if (sc != FTK_OK) return sc;
  const size_t MQ2 = static_cast<size_t>(p->M) * p->two_Q;
  const ChunkLayout L = chunk_layout(p, work, ib, tb, tpack);
  const bool shared = tpack > tb;  // all templates packed once; chunks run image block by image block
  if (shared) {
    const ftk_status st = step1_pack_all_templates(p, precision, b, NT, L.tbuf, s);
    if (st != FTK_OK) return st;
  }
  struct Chunk {
    int i0, ni, j0, nj;
    bool first;  // first chunk of its template block (per-block packs) or of its image block (shared)
  };
  std::vector<Chunk> chunks;
  if (shared) {
    for (int i0 = 0; i0 < NI; i0 += static_cast<int>(ib))
      for (int j0 = 0; j0 < NT; j0 += static_cast<int>(tb))
        chunks.push_back({i0, static_cast<int>(std::min<long long>(ib, NI - i0)), j0,
                          static_cast<int>(std::min<long long>(tb, NT - j0)), j0 == 0});
  } else {
    for (int j0 = 0; j0 < NT; j0 += static_cast<int>(tb)) {
      const int nj = static_cast<int>(std::min<long long>(tb, NT - j0));
      for (int i0 = 0; i0 < NI; i0 += static_cast<int>(ib))
        chunks.push_back({i0, static_cast<int>(std::min<long long>(ib, NI - i0)), j0, nj, i0 == 0});
    }
  }
  for (const Chunk& c : chunks) {
    ftk_status st = tc_run_chunk(p, precision, a + c.i0 * MQ2, c.ni, b + c.j0 * MQ2, c.nj, c.i0, c.j0, NT,
                                 !shared && c.first, L, d_scores, d_keys, rec, s, shared, !shared || c.first);
    if (st != FTK_OK) return st;
    if (rec.wide && d_keys)
      FTK_LAUNCH(p, kKBestMerge, s, launch_best_merge(p, d_keys, c.i0, c.ni, c.j0, nullptr, 0, rec, false, s));
  }
  return FTK_OK;
}

size_t tc_shortlist_bytes(const ftk_plan_s* p, int ni, int K, int NT) {
  return shortlist_chunk_bytes(p, ni, K) + (step1_tc_supported(p) ? al(step1_all_template_bytes(p, NT)) : 0);
}

ftk_status tc_run_shortlist(ftk_plan_s* p, int precision, const float2* a, int NI, const float2* b, int NT,
                            const int* list, int K, const float2* center, float window, unsigned long long* d_keys,
                            const BestRecords& rec, char* work, size_t work_bytes, cudaStream_t s) {
  if (!p->tc.d_Yhi) return FTK_ERR_UNSUPPORTED;
  uint16_t* tall = nullptr;
  if (step1_tc_supported(p)) {  // the whole template set, packed once, at the front of the workspace
    const size_t tb = al(step1_all_template_bytes(p, NT));
    if (tb > work_bytes) return FTK_ERR_NOMEM;
    tall = reinterpret_cast<uint16_t*>(work);
    work += tb;
    work_bytes -= tb;
    ftk_status st0 = step1_pack_all_templates(p, precision, b, NT, tall, s);
    if (st0 != FTK_OK) return st0;
  }
  if (shortlist_chunk_bytes(p, 1, K) > work_bytes) return FTK_ERR_NOMEM;
  long long ib = 1;
  while (ib < NI && ib < 65535 && shortlist_chunk_bytes(p, std::min<long long>({NI, ib * 2, 65535}), K) <= work_bytes)
    ib = std::min<long long>({NI, ib * 2, 65535});
  const int x3 = op_mode(precision);
  const int Kpad = p->tc.Kpad;
  const size_t MQ2 = static_cast<size_t>(p->M) * p->two_Q;
  for (int i0 = 0; i0 < NI; i0 += static_cast<int>(ib)) {
    const int ni = static_cast<int>(std::min<long long>(ib, NI - i0));
    const long long pairs = static_cast<long long>(ni) * K;
    const long long R = pairs * p->n_rot;
    if (R > 0x7FFFFFFFLL) return FTK_ERR_UNSUPPORTED;
    const int n_tiles = static_cast<int>((R + kRows - 1) / kRows);
    char* w = work;
    float2* zbuf = reinterpret_cast<float2*>(w);
    w += al(static_cast<size_t>(pairs) * ((p->Hh + 1) & ~1) * p->two_Q * sizeof(float2));
    uint16_t* zhi = reinterpret_cast<uint16_t*>(w);
    w += al(static_cast<size_t>(n_tiles) * kRows * Kpad * sizeof(uint16_t));
    uint16_t* zlo = reinterpret_cast<uint16_t*>(w);
    w += al(static_cast<size_t>(n_tiles) * kRows * Kpad * sizeof(uint16_t));
    if (step1_tc_supported(p)) {
      uint16_t* tbuf = reinterpret_cast<uint16_t*>(w);
      w += al(static_cast<size_t>(ni) * step1_list_template_bytes(p, K));
      uint16_t* ibuf = reinterpret_cast<uint16_t*>(w);
      ftk_status st1 = step1_tc_run_list(p, precision, a + i0 * MQ2, ni, tall, NT, list + static_cast<size_t>(i0) * K,
                                         K, zbuf, tbuf, ibuf, s);
      if (st1 != FTK_OK) return st1;
    } else {
      FTK_LAUNCH(p, kKStep1Simt, s, launch_step1_list_tc(p, a + i0 * MQ2, ni, b, K, list + static_cast<size_t>(i0) * K,
                                                         zbuf, s));
    }
    // wide pose indices: keys by list position, merged into the records after each chunk
    const int key_pos = rec.wide ? 1 : 0;
    const bool fused = step23_supported(p, precision);
    if (fused || step23c_supported(p, precision)) {  // Steps 2-3 fused (in one CTA, or over a cluster)
      ftk_status st = fused ? step23_run(p, precision, zbuf, pairs, K, i0, 0, d_keys, list, center, window, 0,
                                         key_pos, s)
                            : step23c_run(p, precision, zbuf, pairs, K, i0, 0, d_keys, list, center, window, 0,
                                          key_pos, s);
      if (st != FTK_OK) return st;
      if (rec.wide) FTK_LAUNCH(p, kKBestMerge, s, launch_best_merge(p, d_keys, i0, ni, 0, list, K, rec, false, s));
      continue;
    }
    const long long blocks = pairs * (Kpad / 16);
    if (blocks > 0x7FFFFFFFLL) return FTK_ERR_UNSUPPORTED;
    ftk_status st = launch_fft_pack(p, zbuf, blocks, Kpad, zhi, zlo, x3, s);
    if (st != FTK_OK) return st;
    Step3Args args = step3_args(p, x3, zhi, zlo, n_tiles, R, K, i0, 0, NT);
    args.keys = d_keys;
    args.list = list;
    args.center = center;
    args.window = window;
    args.key_pos = key_pos;
    st = launch_step3(p, args, s);
    if (st != FTK_OK) return st;
    if (rec.wide) FTK_LAUNCH(p, kKBestMerge, s, launch_best_merge(p, d_keys, i0, ni, 0, list, K, rec, false, s));
  }
  return FTK_OK;
}

}  // namespace ftk
