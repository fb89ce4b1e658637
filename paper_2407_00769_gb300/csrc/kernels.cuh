// Device kernels of the contraction library: launch wrappers and the
// parameter blocks the host fills.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "internal.h"

namespace tn {

// Bit-permute transpose of a tensor of 2^rank elements (all modes dim 2).
// The host precomputes the tile decomposition (see make_perm_params).
struct PermParams {
    int32_t rank;
    int32_t tile_bits;      // bits of the element index covered by one tile
    int32_t lin;            // low input bits read contiguously
    int32_t lout;           // low output bits written contiguously
    int32_t n_outer;        // rank - tile_bits
    int32_t pad_;
    int64_t rd_hi_off[32];  // read-order high bits -> input offset
    int32_t wr_lo_e[32];    // write-order low bits -> read-order index bits
    int32_t wr_hi_e[32];    // write-order high bits -> read-order index bits
    int64_t wr_hi_off[32];  // write-order high bits -> output offset
    int8_t outer_in[kMaxRank], outer_out[kMaxRank];  // tile-id bit k -> in/out position
};

// perm: output mode i (outermost first) = input mode perm[i].
PermParams make_perm_params(int rank, const int32_t *perm);

struct ScaleRef {          // power-of-two scaling state (complex-half)
    const float *tmax;     // per-tensor max |component| of stored values
    int32_t *texp;         // per-tensor exponent E: true value = stored * 2^-E
    int32_t meta_a, meta_b, meta_c;
    int32_t fixed_exp;     // used when tmax == nullptr (tests): e = fixed_exp
    float *out_max;        // where the epilogue records max |C| (atomicMax)
    int32_t headroom;      // added to the bound-based exponent (calibrated per step)
    int32_t *err;          // bit 2 set when a stored value overflowed (inf)
    int32_t scale_off;     // 1: every exponent e = 0 (tn_plan_opts.no_scaling)
};

cudaError_t launch_leaf_prep(const LeafJob *d_jobs, int count, const double2 *d_store, char *ws,
                             int dtype, int64_t slice_base, float *tmax, int32_t *texp,
                             cudaStream_t s);
cudaError_t launch_permute(const void *in, void *out, const PermParams &pp, int elem_bytes,
                           cudaStream_t s);
// za / zb (device int32[batch], nullable): the A / B chunk of each batch
// entry (sparse-state gathers); NULL: the entry itself (times sa / sb).
cudaError_t launch_gemm_rows_c64(const float2 *A, const float2 *B, float2 *C, int lm, int ln,
                                 int lk, int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                                 cudaStream_t s, const int32_t *za = nullptr, const int32_t *zb = nullptr);
cudaError_t launch_gemm_tiled_c64(const float2 *A, const float2 *B, float2 *C, int lm, int ln,
                                  int lk, int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                                  int tile, cudaStream_t s, const int32_t *za = nullptr,
                                  const int32_t *zb = nullptr);
cudaError_t launch_gemm_rows_lp(int dtype, const void *A, const void *B, void *C, int lm, int ln,
                                int lk, int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                                const ScaleRef &sr, cudaStream_t s);
cudaError_t launch_bprep(int dtype, const void *B, void *Bp, int lk, int ln, int64_t batch, int np,
                         cudaStream_t s);
// B in any mode order -> B' in one pass (perm: output mode i of the
// [batch][N][K] order = stored mode perm[i]); complex-half only.
// tb = 0: B is complex64, rounded here to `dtype`, and the rounding's
// compensation factor 1/(1 + alpha) is written to *corr.
// and B is first scaled by an exact 2^s that brings its recorded maximum
// (tmax[meta_src]) near 2^12; B' gets tmax[meta_dst] and texp[meta_dst] =
// texp[meta_src] + s.
// scale_off = 1: no 2^s (s = 0; tn_plan_opts.no_scaling).
// scratch (tb = 0, nullable): bprep_c64_scratch_bytes() of device memory for
// the multi-block build; NULL: one block.
cudaError_t launch_bprep_perm(const void *B, void *Bp, int rank, const int32_t *perm, int lk, int ln,
                              int lb, int np, int tb, int dtype, double2 *corr, float *tmax,
                              int32_t *texp, int meta_src, int meta_dst, cudaStream_t s,
                              int scale_off = 0, void *scratch = nullptr);
size_t bprep_c64_scratch_bytes();
// complex64 on the tensor cores (TcGemmDesc::x3): x -> hi + lo parts of n
// FP32 values (n a multiple of 4, 16-byte aligned), and complex64 B
// [batch][K][N] -> the FP32 B' [batch][np][2K] of Eq. 6 as hi and lo parts
cudaError_t launch_split_tf32(const void *x, void *hi, void *lo, int64_t n, cudaStream_t s);
cudaError_t launch_bprep_x3(const void *B, void *bh, void *bl, int lk, int ln, int64_t batch, int np, cudaStream_t s);
cudaError_t launch_gemm_rows_mixed(int dtype, int ta, int tb, int tc, const void *A, const void *B,
                                   void *C, int lm, int ln, int lk, int64_t batch, int64_t sa,
                                   int64_t sb, int64_t sc, const ScaleRef &sr, cudaStream_t s,
                                   const int32_t *za = nullptr, const int32_t *zb = nullptr);
// stepcorr / n_steps: per-step rounding compensation factors of a
// complex-half plan (n_steps = 0: none).  split_val: the values of the
// op's split outputs (recomputation) for this pass, as amplitude-index bits;
// only the 2^(n_open - n_split) amplitudes with those bits are written.
cudaError_t launch_slice_sum(const void *F, int dtype, const SumOp &op, double2 *amps, int n_open,
                             int t_lo, int t_hi, int overwrite, const int32_t *texp,
                             const double2 *stepcorr, int n_steps, uint64_t split_val, cudaStream_t s);
cudaError_t launch_metrics(const double2 *r, const double2 *b, int64_t n, double *d_out5,
                           double *d_partials, int n_blocks, cudaStream_t s);
cudaError_t launch_topk(const double2 *amps, int64_t n, int k, int64_t *d_idx, double *d_prob,
                        cudaStream_t s);
// Top-k of n amplitudes in the order (|amp|^2 descending, index ascending):
// the one-block kernel above while k * n <= 2^22, else a multi-block radix
// select (O(n) reads per pass, 8 passes), a collection of the k entries and
// a bitonic sort.  scratch: topk_scratch_bytes(n, k) bytes of device memory
// (0: none needed); d_idx / d_prob: device, k entries each.
bool topk_one_block(int64_t n, int64_t k);
size_t topk_scratch_bytes(int64_t n, int64_t k);
cudaError_t launch_topk_select(const double2 *amps, int64_t n, int64_t k, void *scratch, int64_t *d_idx,
                               double *d_prob, cudaStream_t s);

// tcgen05 GEMM (complex-half as real, Eq. 5-6).  Tensor maps are encoded
// by the host (tc_gemm.cu).
struct TcGemmDesc {
    int dtype;             // TN_F16 | TN_BF16
    const void *A;         // [batch_a][M][2K] real
    const void *Bp;        // [batch_b][np][2K] real (padded B')
    void *C;               // [batch][M][N] complex-half
    int lm, ln, lk;
    int64_t batch;
    int batch_a, batch_b;  // 1: operand has the batch dim, 0: broadcast
    int np;                // padded real columns of B' (>= 16, power of 2)
    int withhold = 0;      // self-test: the TMA producer issues nothing
    int bn = 0;            // N-tile width in real columns (0: min(np, 256))
    int gm = 0;            // m tiles per raster group (0: from the L2 budget)
    int out_c64 = 0;       // write C as complex64 (no rounding, exponent e = 0)
    float *partial = nullptr;  // tc_split_bytes() of FP32 partials when tc_split() > 1
    int fp8 = 0;           // A and B' are E4M3 bytes (kind::f8f6f4), K >= 64
    // sparse-state gathers: per batch entry the A chunk, B' chunk and output
    // chunk (device int32[batch], < 0 output: not stored); depth_a/depth_b:
    // chunks held by A and B' (0: from batch_a / batch_b).  K <= 2^15.
    const int32_t *za = nullptr, *zb = nullptr, *zc = nullptr;
    int64_t depth_a = 0, depth_b = 0;
    // padded 2-D index: gather_r B' chunks side by side per N tile (bn =
    // gather_r * np), zb/zc indexed [batch][m_r]; 0: one chunk per entry
    int gather_r = 0, m_r = 0;
    // > 0: write C in a permuted mode order (bit i of the natural element
    // index -> bit out_dpos[i]; bits 0..2 unchanged, N >= 8, K <= 2^15)
    int out_rank = 0;
    int8_t out_dpos[40] = {};
    // 1: run on CTA pairs (256-row tiles, cluster of 2) where the shape allows
    int pair = 0;
    // 1: 64-byte K chunks (FP16/BF16, 1-CTA tiles): a deeper ring
    int half_k = 0;
    // 1: complex64 operands on the tensor cores (kind::tf32, three MMAs per
    // K slice): A / Bp hold the TF32 "hi" parts (FP32 words with 13 low
    // mantissa bits clear) and A2 / Bp2 the remainders, all FP32 in the
    // layouts of A and B'; C complex64 (out_c64 = 1); 1-CTA tiles, N tile <=
    // 128, no gathers
    int x3 = 0;
    const void *A2 = nullptr, *Bp2 = nullptr;
    // 1: complex-half results through a per-warp staging area in shared
    // memory, every store instruction writing whole 32-byte sectors
    // (tc_store_block; 1-CTA and pair kernels)
    int staged = 0;
    // 1: keep each walker's B' slice resident in shared memory (short-K
    // steps, gemm_tc_bres_kernel) where the step allows it
    int bres = 0;
    // with bres: write C tiles staged in shared memory with TMA stores
    // (complex-half C in natural order, N tiles of 64-column multiples)
    int tma_store = 0;
};

// E4M3 operands of an FP8 tensor-core step: n_pairs FP16/BF16 values pairs
// (a complex-half tensor, or B' read as pairs of reals) -> E4M3 pairs scaled
// by 2^s, s chosen on the device from tmax[meta_src] so that the largest
// magnitude lands in (224, 448] (E4M3's largest finite value is 448); writes
// tmax[meta_dst] (atomic max, slot zeroed beforehand) and texp[meta_dst] =
// texp[meta_src] + s.  Round to nearest even, saturating.
cudaError_t launch_quant_e4m3(const void *src, void *dst, int64_t n_pairs, int dtype, float *tmax,
                              int32_t *texp, int meta_src, int meta_dst, cudaStream_t s);
// B [batch][K][N] complex E4M3 -> B' [batch][np][2K] E4M3 (Eq. 6 padding)
cudaError_t launch_bprep_e4m3(const void *B, void *Bp, int lk, int ln, int64_t batch, int np,
                              cudaStream_t s);
bool tc_gemm_supported_fp8(int lk, int ln);

// Split-K: the tensor cores' FP32 accumulation over very long K drifts
// (error growing with K), so a step with K > 2^kSplitLog2K complex is cut
// into parts of that length, each accumulated separately in TMEM, and the
// parts are added here in FP64, in part order (deterministic), then scaled
// and rounded like the single-part epilogue.
constexpr int kSplitLog2K = 15;
int tc_split(int lm, int ln, int lk, int64_t batch);
size_t tc_split_bytes(int lm, int ln, int lk, int64_t batch);
cudaError_t launch_splitk_reduce(const float *partial, int split, void *C, int out_c64, int dtype,
                                 int64_t batch, int lm, int ln, int lk, const ScaleRef &sr,
                                 cudaStream_t s);

// Tile configuration of a tensor-core step: (bn, gm) packed as
// bn_code | gm_code << 4 (code 0 = automatic choice).
constexpr int kTcBn[5] = {0, 256, 128, 64, 32};
constexpr int kTcGm[6] = {0, 4, 8, 16, 32, 64};
inline int tc_tile_bn(int tile) { return kTcBn[(tile & 15) < 5 ? (tile & 15) : 0]; }
inline int tc_tile_gm(int tile) { return kTcGm[((tile >> 4) & 15) < 6 ? ((tile >> 4) & 15) : 0]; }
// The (BN, raster group) codes a tensor-core launch with tile code `tile`
// really uses for N = 2^ln (tile 0 and explicit codes may coincide).
int tc_effective_tile(int tile, int ln);
bool tc_gemm_supported(int lk, int ln);
// whether a step of this shape can run on the B'-resident kernel with an N
// tile of bn real columns (1-CTA FP16/BF16, one K part, no gathers, the whole
// K of a B' slice within 64 KiB)
bool tc_bres_eligible(int lm, int ln, int lk, int64_t batch, int bn, int fp8, int gathered);
// the same with the C tiles written by TMA stores (complex-half C in natural
// order, bn a multiple of 64, room for two staged C tiles)
bool tc_bres_store_eligible(int lm, int ln, int lk, int64_t batch, int bn);
cudaError_t launch_gemm_tc(const TcGemmDesc &d, const ScaleRef &sr, int32_t *d_err,
                           cudaStream_t s);
int tc_num_sms();
cudaError_t tc_prepare();

}  // namespace tn
