// Tensor-core (tcgen05) pair engine: interface used by the C-ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ftk_internal.h"

namespace ftk {

// Operand mode of the tensor-core kernels for an ftk_precision (tc_ptx.cuh OperandMode:
// 0 = one BF16 term, 1 = BF16x3, 2 = one FP16 term).
inline int op_mode(int precision) {
  return precision == FTK_BF16X3 ? 1 : (precision == FTK_FP16 ? 2 : 0);
}

// Whether the plan's sizes fit the tcgen05 kernels.
bool tc_supported(const ftk_plan_s* p);
// Scratch (bytes, excluding per-image keys) of the tensor path: the smallest that
// works and a size that allows large chunks.
void tc_workspace(const ftk_plan_s* p, int NI, int NT, size_t* min_bytes, size_t* good_bytes);
// Builds/frees the split-precision shift-factor tables.
cudaError_t tc_build_tables(ftk_plan_s* p, const std::vector<float2>& Y);
void tc_free_tables(ftk_plan_s* p);
// Steps 1-3 over all NI x NT pairs, chunked to fit work_bytes. With rec.wide the keys of
// each chunk count templates from the chunk's first one and are merged into rec after it.
ftk_status tc_run_all(ftk_plan_s* p, int precision, const float2* a, int NI, const float2* b, int NT, float* d_scores,
                      unsigned long long* d_keys, const BestRecords& rec, char* work, size_t work_bytes,
                      cudaStream_t s);

// Steps 1-3 over per-image template lists list [NI][K] (entries in range) with optional
// shift windows: Step 1 on tensor cores in list mode (each image against its own tile of
// listed templates), Steps 2-3 as above. With rec.wide the keys count list positions and
// are merged into rec after each chunk of images.
size_t tc_shortlist_bytes(const ftk_plan_s* p, int ni, int K, int NT);
ftk_status tc_run_shortlist(ftk_plan_s* p, int precision, const float2* a, int NI, const float2* b, int NT,
                            const int* list, int K, const float2* center, float window, unsigned long long* d_keys,
                            const BestRecords& rec, char* work, size_t work_bytes, cudaStream_t s);

// Steps 2-3 fused with the best-pose epilogue (k_step23_tc.cu): whether the plan's
// sizes fit (and the "step23" knob allows it), and the run over `pairs` pairs of
// Zhat [pair][2Q][Hs] (pair = il * nj + jl; template j0 + jl, or list[i][jl]); the template
// part of a key's pose index is j - jbase, or jl with key_pos.
bool step23_supported(const ftk_plan_s* p, int precision);
ftk_status step23_run(ftk_plan_s* p, int precision, const float2* zhat, long long pairs, int nj, int i0, int j0,
                      unsigned long long* keys, const int* list, const float2* center, float window, int jbase,
                      int key_pos, cudaStream_t s);

// Steps 2-3 fused over a cluster of n_groups CTAs for 2Q = 128 R, R = 2..4 (k_step23c_tc.cu):
// each CTA holds one shift group of the Step-3 B operand; the DFT over q of each pair is
// computed once per cluster, K slice by K slice, and shared through the cluster's shared
// memory. Same arguments and results as step23_run.
bool step23c_supported(ftk_plan_s* p, int precision);
ftk_status step23c_run(ftk_plan_s* p, int precision, const float2* zhat, long long pairs, int nj, int i0, int j0,
                       unsigned long long* keys, const int* list, const float2* center, float window, int jbase,
                       int key_pos, cudaStream_t s);

// Polar transform on tensor cores (k_transform_tc.cu).
bool xform_tc_supported(const ftk_plan_s* p);
cudaError_t xform_build_tables(ftk_plan_s* p, const std::vector<double>& ey_re, const std::vector<double>& ey_im);
cudaError_t xform_alloc_scratch(ftk_plan_s* p);
void xform_free_tables(ftk_plan_s* p);
ftk_status xform_run(ftk_plan_s* p, const float* d_images, int B, float2* d_out, cudaStream_t s);

// Step 1 on tensor cores (k_tc_step1.cu).
bool step1_tc_supported(const ftk_plan_s* p);
size_t step1_image_bytes(const ftk_plan_s* p);
size_t step1_template_row_bytes(const ftk_plan_s* p);
ftk_status step1_tc_run(ftk_plan_s* p, int precision, const float2* a, int ni, const float2* b, int nj, float2* zhat,
                        uint16_t* tbuf, uint16_t* ibuf, bool pack_templates, cudaStream_t s);
// Step 1 of templates [128 jt0, 128 jt0 + nj) of a set of NT templates packed once as a whole
// (step1_pack_all_templates into `tall`); the ni images are packed into ibuf first when
// pack_images, else ibuf already holds them (an earlier block of the same images).
ftk_status step1_tc_run_block(ftk_plan_s* p, int precision, const float2* a, int ni, int nj, int jt0, int NT,
                              const uint16_t* tall, float2* zhat, uint16_t* ibuf, bool pack_images, cudaStream_t s);
// Step 1 of per-image template lists list [ni][K] (entries in range): the templates of each
// image are packed per image and multiplied with that image only; Zhat [i * K + jj][q][zeta].
// The templates are packed once (step1_pack_all_templates into `tall`) and each image's
// tiles gathered from that pack.
size_t step1_list_template_bytes(const ftk_plan_s* p, int K);  // per image
size_t step1_all_template_bytes(const ftk_plan_s* p, int NT);
ftk_status step1_pack_all_templates(ftk_plan_s* p, int precision, const float2* b, int NT, uint16_t* tall,
                                    cudaStream_t s);
ftk_status step1_tc_run_list(ftk_plan_s* p, int precision, const float2* a, int ni, const uint16_t* tall, int NT,
                             const int* list, int K, float2* zhat, uint16_t* tbuf, uint16_t* ibuf, cudaStream_t s);

}  // namespace ftk
