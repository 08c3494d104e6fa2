// Internal declarations shared by the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ftk.h"  // include/ftk.h (on the include path)

namespace ftk {

constexpr int kMaxRadix = 8;

// Bits of the plan's device error word (read and cleared by ftk_stream_check).
constexpr int kErrTimeout = 1;  // a bounded wait gave up
constexpr int kErrIndex = 2;    // a device-side index argument was out of range

// Radix schedule of a length-L Stockham FFT (L = 2^a 3^b).
struct FftSchedule {
  int L = 0;
  int n = 0;
  int radix[12] = {0};
};
FftSchedule make_fft_schedule(int L);

// Kernel identifiers for the launch profiler (ftk_profile_*).
enum KernelId {
  kKPolar = 0,
  kKFftRows,
  kKStep1Simt,
  kKStep3Simt,
  kKBestInit,
  kKBestFinalize,
  kKStep1Tc,
  kKFftPack,
  kKStep3Tc,
  kKPackTemplates,
  kKPolarTc,
  kKPackPixels,
  kKStep23Tc,
  kKBestMerge,
  kKStep23cTc,
  kKNumKernels
};
const char* kernel_name(int id);

// CUDA-event timing of every launch of each kernel on its own stream, enabled
// between ftk_profile_begin and ftk_profile_end.
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pending_start[kKNumKernels];
  std::vector<cudaEvent_t> pending_stop[kKNumKernels];
  double total_ms[kKNumKernels] = {0};
  long long count[kKNumKernels] = {0};
};

// Device-side tables of the tensor-core path (filled at plan creation).
// Launch-shape knobs of the tensor path (ftk_plan_tune); 0 = library default.
struct TcTuning {
  int step3_group_max = 0;   // upper bound on the shift-group size G (multiple of 16)
  int step3_a_stages = 0;    // A-tile stages of Step 3 (1..4)
  int step1_stages = 0;      // operand stages of Step 1 (2..8)
  int step1_ctas_per_sm = 0; // work units per SM that Step 1 aims for (1..8)
  int fft_lanes = 0;         // Step 2 + pack: 0 = lanes per transform by length, 32 = one warp each
  int step23 = 1;            // best-pose search: 1 = fused Steps 2-3 where they fit, 0 = separate kernels
  int cluster23 = 0;         // 1: Steps 2-3 fused over a CTA cluster where 2Q = 128 R (with step23 = 1)
  int checks = 0;            // 1: the fused Steps 2-3 check every index (latch kErrIndex, skip the access)
};

// Tensor-core polar transform: the Ey^T operand (packed once per plan) and the
// plan-owned scratch for packed pixels (pix_images images per launch).
struct XfTables {
  uint16_t* d_ehi = nullptr;
  uint16_t* d_elo = nullptr;
  uint16_t* d_pix = nullptr;
  int pix_images = 0;
  bool use_simt = false;  // the FP32 SIMT transform instead (tuning knob "transform")
};

struct TcTables {
  int Kpad = 0;          // 2*H_half rounded up to a multiple of 16 (MMA K)
  int G = 0;             // shifts per group (MMA N of Step 3), multiple of 16, <= 256
  int n_groups = 0;      // shift groups; Y rows padded to n_groups * G
  int nsa = 2;           // A-tile stages of Step 3
  uint16_t* d_Yhi = nullptr;  // [n_groups * G][Kpad] bf16: Y' split, K-major core-matrix layout
  uint16_t* d_Ylo = nullptr;  // [n_groups * G][Kpad] bf16
  int n_mt = 0;               // 128-shift tiles of the fused Steps 2-3
  uint16_t* d_Yrhi = nullptr; // [n_mt * 128][Kpad] bf16 hi, row-major (the fused kernel's TMEM operand)
  uint16_t* d_Yrlo = nullptr; // [n_mt * 128][Kpad] bf16 lo
  uint16_t* d_Yh16 = nullptr; // as d_Yhi, FP16 (precision FTK_FP16)
  uint16_t* d_Yr16 = nullptr; // as d_Yrhi, FP16
  // clusters of n_groups CTAs that the cluster-fused Steps 2-3 can run at once, per operand
  // mode (-1: not yet asked; set again whenever the tables are rebuilt)
  int max_clusters[3] = {-1, -1, -1};
};

}  // namespace ftk

struct ftk_plan_s {
  int device = 0;
  int n = 0, M = 0, two_Q = 0, Q = 0, N = 0;  // N = rows of the shift factors = N_shift * n_tau
  int N_shift = 0, n_tau = 1;                   // shifts, CTF defocus values (1 without CTF)
  double K = 0, W = 0, eps = 0, dx = 0;
  int H = 0;       // sum over all l of H_l
  int Hh = 0;      // terms with l >= 0
  int L = 0;       // largest l with H_l > 0
  std::vector<int> h_l;          // [Hh]
  std::vector<double> h_sigma;   // [Hh]
  std::vector<double> h_k, h_w;  // [M]
  ftk::FftSchedule fft;          // length 2Q
  // device tables
  float* d_G = nullptr;     // [Hh][M]  2 pi w_m G_zeta(k_m)
  int* d_l = nullptr;       // [Hh]
  float2* d_Y = nullptr;    // [N][Hh]  c_zeta Y_zeta(delta_s), c = 1 (l = 0) or 2 (l > 0)
  float2* d_shifts = nullptr;  // [N] shifts in pixels
  float2* d_Ex = nullptr;   // [n][M*Q] exp(-i k_m cos(psi_p) x_i), p < Q
  float2* d_Ey = nullptr;   // [n][M*Q] exp(-i k_m sin(psi_p) y_j), p < Q
  float2* d_tw = nullptr;   // [2Q] exp(-2 pi i t / 2Q)
  // rotation grid: n_rot = 2Q (Section 3.2) or a multiple of it (Step 2 zero-padded)
  int n_rot = 0;
  float2* d_tw_rot = nullptr;  // [n_rot] exp(-2 pi i t / n_rot) when n_rot != 2Q
  int* d_err = nullptr;     // device error latch: bit kErrTimeout (bounded waits), bit kErrIndex
  ftk::TcTables tc;
  ftk::XfTables xf;
  ftk::TcTuning tune;
  std::vector<float2> h_Y;       // [N][Hh] shift factors (kept to rebuild the split tables)
  std::vector<float> h_G;        // [Hh][M] radial factors 2 pi w_m G_zeta(k_m) (kept for ftk_plan_save)
  std::vector<double> h_shifts;  // [N_shift][2] shifts in pixels
  std::vector<double> h_taus;    // CTF defocus values (empty without CTF)
  double phase = 0;              // CTF phase
  double decay = 0;              // spectral weight of the modal SVDs (0: plain weights)
  long long launches = 0;
  ftk::Profiler prof;
};

namespace ftk {

// The plan's device tables live on the device that was current when it was created (or
// loaded); calls that launch work on them need that device current (else FTK_ERR_ARG).
bool on_plan_device(const ftk_plan_s* p);

void prof_start(ftk_plan_s* p, int id, cudaStream_t s);
void prof_stop(ftk_plan_s* p, int id, cudaStream_t s);

}  // namespace ftk

// Launch a kernel through its launcher, time it when profiling, count it.
#define FTK_LAUNCH(p, id, s, call)                       \
  do {                                                   \
    ftk::prof_start((p), (id), (s));                     \
    cudaError_t e_ = (call);                             \
    ftk::prof_stop((p), (id), (s));                      \
    (p)->launches++;                                     \
    if (e_ != cudaSuccess) return FTK_ERR_CUDA;          \
  } while (0)

namespace ftk {

// ---- kernel launchers (return cudaGetLastError()) ----
cudaError_t launch_polar_transform(const ftk_plan_s* p, const float* d_images, int B, float2* d_out,
                                   cudaStream_t s);
cudaError_t launch_fft_rows(const ftk_plan_s* p, float2* d_rows, long long nrows, float scale,
                            cudaStream_t s);

// FP32 SIMT pair engine
// d_list_chunk: per-image template lists of this chunk's images ([ni][nj], NULL = all templates)
cudaError_t launch_step1_simt(const ftk_plan_s* p, const float2* d_a, int ni, const float2* d_b,
                              int nj, float2* d_zhat, cudaStream_t s, const int* d_list_chunk = nullptr);
// Step 1 of per-image template lists ([ni][nj], every entry in range) into the tensor-core
// layout Zhat [pair][q][zeta] (row stride Hh rounded up to even)
cudaError_t launch_step1_list_tc(const ftk_plan_s* p, const float2* d_a, int ni, const float2* d_b, int nj,
                                 const int* d_list_chunk, float2* d_zhat, cudaStream_t s);
// d_list: per-image template lists indexed by the global image ([NI][nj]); d_center: per-image
// shift-window centres in pixels ([NI]), NULL = every shift; jbase / key_pos: the template
// part of a key's pose index is j - jbase (key_pos = 0) or the list position (key_pos = 1)
cudaError_t launch_step3_simt(const ftk_plan_s* p, const float2* d_z, int ni, int nj, int i0, int j0,
                              int NT, float* d_scores, unsigned long long* d_keys, cudaStream_t s,
                              const int* d_list = nullptr, const float2* d_center = nullptr, float window = 0.f,
                              int jbase = 0, int key_pos = 0);
// copies a [n] template list into d_out with indices outside [0, NT) replaced by 0 (latches kErrIndex)
cudaError_t launch_sanitize_list(const ftk_plan_s* p, const int* d_in, long long n, int NT, int* d_out,
                                 cudaStream_t s);
cudaError_t launch_best_init(unsigned long long* d_keys, int NI, cudaStream_t s);
cudaError_t launch_best_finalize(const ftk_plan_s* p, const unsigned long long* d_keys, int NI,
                                 int* d_tpl, int* d_rot, int* d_shift, float* d_score, cudaStream_t s);

// Best-pose searches whose pose index NT * R * N reaches 2^32 ("wide"): each chunk's keys
// count templates from the chunk's first template (or by list position) and are merged
// after the chunk into per-image records kept in the caller's outputs.
struct BestRecords {
  bool wide = false;
  int* tpl = nullptr;
  int* rot = nullptr;
  int* shift = nullptr;
  float* score = nullptr;
};
inline bool pose_index_wide(long long NT, int R, int N) {
  return static_cast<double>(NT) * R * N >= 4294967295.0;
}
cudaError_t launch_best_init_records(unsigned long long* d_keys, int NI, int* d_tpl, int* d_rot, int* d_shift,
                                     float* d_score, cudaStream_t s);
cudaError_t launch_best_merge(const ftk_plan_s* p, unsigned long long* d_keys, int i0, int ni, int jbase,
                              const int* d_list, int K, const BestRecords& rec, bool last, cudaStream_t s);

}  // namespace ftk
