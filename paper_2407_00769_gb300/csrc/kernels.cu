// SIMT kernels: leaf preparation (slice decoding), bit-permute transpose,
// complex GEMMs on CUDA cores, B padding for the tensor-core path, the FP64
// cross-slice sum, FP64 reductions and top-k post-selection.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "bodies.cuh"
#include "kernels.cuh"

namespace tn {

// ------------------------------------------------------------- leaf prep --
// One block (one warp) per leaf: leaf_warp_body (slice decoding and the
// complex128 -> complex64 conversion).
__global__ void leaf_prep_kernel(const LeafJob *jobs, const double2 *store, char *ws,
                                 int64_t slice_base, float *tmax, int32_t *texp) {
    leaf_warp_body(jobs[blockIdx.x], store, ws, slice_base, tmax, texp, threadIdx.x);
}

cudaError_t launch_leaf_prep(const LeafJob *d_jobs, int count, const double2 *d_store, char *ws,
                             int dtype, int64_t slice_base, float *tmax, int32_t *texp,
                             cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    // leaves are stored complex64 in every plan; complex-half plans record
    // each leaf's maximum for the scaling of the steps that consume it
    leaf_prep_kernel<<<count, 32, 0, s>>>(d_jobs, d_store, ws, slice_base,
                                          dtype == TN_C64 ? nullptr : tmax, texp);
    return cudaGetLastError();
}

// --------------------------------------------------------------- permute --
// Tile = a set of input index bits (the low `lin` input bits plus the input
// positions of the low `lout` output bits, topped up to `tile_bits`).  A
// block reads its tile in input order (coalesced), stages it in shared
// memory, and writes it in output order (coalesced).  The other bits come
// from the block id.  Pure data movement: bit-exact.
PermParams make_perm_params(int r, const int32_t *perm) {
    PermParams p;
    std::memset(&p, 0, sizeof(p));
    p.rank = r;
    // out_of_in[b] = output bit position of input bit position b (LSB = 0)
    int out_of_in[kMaxRank], in_of_out[kMaxRank];
    for (int i = 0; i < r; ++i) {
        const int in_bit = r - 1 - perm[i], out_bit = r - 1 - i;
        out_of_in[in_bit] = out_bit;
        in_of_out[out_bit] = in_bit;
    }
    const int tb = std::min(10, r);
    p.lin = std::min(5, r);
    p.lout = std::min(5, r);
    bool in_tile[kMaxRank] = {false};
    for (int b = 0; b < p.lin; ++b) in_tile[b] = true;
    for (int j = 0; j < p.lout; ++j) in_tile[in_of_out[j]] = true;
    int count = 0;
    for (int b = 0; b < r; ++b) count += in_tile[b];
    for (int b = 0; b < r && count < tb; ++b)
        if (!in_tile[b]) { in_tile[b] = true; ++count; }
    p.tile_bits = count;
    // read order: e bit i < lin -> input bit i; e bit lin+k -> hi_pos[k]
    int hi_pos[kMaxRank], n_hi = 0;
    int e_bit_of_in[kMaxRank];
    for (int b = 0; b < r; ++b) e_bit_of_in[b] = -1;
    for (int b = 0; b < p.lin; ++b) e_bit_of_in[b] = b;
    for (int b = p.lin; b < r; ++b)
        if (in_tile[b]) { e_bit_of_in[b] = p.lin + n_hi; hi_pos[n_hi++] = b; }
    for (int h = 0; h < (1 << n_hi); ++h) {
        int64_t off = 0;
        for (int k = 0; k < n_hi; ++k)
            if ((h >> k) & 1) off |= (int64_t)1 << hi_pos[k];
        p.rd_hi_off[h] = off;
    }
    // write order: f bit j < lout -> output bit j; f bit lout+k -> the k-th
    // remaining tile bit (ascending output position)
    int whi_out[kMaxRank], n_whi = 0;
    for (int ob = p.lout; ob < r; ++ob)
        if (in_tile[in_of_out[ob]]) whi_out[n_whi++] = ob;
    for (int f = 0; f < (1 << p.lout); ++f) {
        int e = 0;
        for (int j = 0; j < p.lout; ++j)
            if ((f >> j) & 1) e |= 1 << e_bit_of_in[in_of_out[j]];
        p.wr_lo_e[f] = e;
    }
    for (int h = 0; h < (1 << n_whi); ++h) {
        int e = 0;
        int64_t off = 0;
        for (int k = 0; k < n_whi; ++k)
            if ((h >> k) & 1) {
                e |= 1 << e_bit_of_in[in_of_out[whi_out[k]]];
                off |= (int64_t)1 << whi_out[k];
            }
        p.wr_hi_e[h] = e;
        p.wr_hi_off[h] = off;
    }
    // outer bits
    int k = 0;
    for (int b = 0; b < r; ++b)
        if (!in_tile[b]) {
            p.outer_in[k] = (int8_t)b;
            p.outer_out[k] = (int8_t)out_of_in[b];
            ++k;
        }
    p.n_outer = k;
    return p;
}

template <typename T>
__global__ void __launch_bounds__(256) permute_kernel(const T *__restrict__ in, T *__restrict__ out,
                                                      const __grid_constant__ PermParams p) {
    __shared__ T tile[1024 + 32];
    permute_tile_body<T, SyncBlock>(in, out, p, blockIdx.x, threadIdx.x, blockDim.x, tile);
}

// Fast path for tensors of rank >= 10 (permute_tiled_body), persistent over
// the tiles; EXPAND writes the padded tensor-core operand B' instead.
template <typename T, bool EXPAND>
__global__ void __launch_bounds__(256) permute_tiled_kernel(const T *__restrict__ in,
                                                            void *__restrict__ out_,
                                                            const __grid_constant__ PermParams p,
                                                            int64_t ntiles, ExpandArgs ex) {
    __shared__ PermTiledSmem<T> sm;
    permute_tiled_body<T, EXPAND, SyncBlock>(in, out_, p, blockIdx.x, ntiles, gridDim.x, ex, threadIdx.x, sm);
}

static int64_t permute_grid(int64_t ntiles) {
    return std::min<int64_t>(ntiles, (int64_t)tc_num_sms() * 8);
}

cudaError_t launch_permute(const void *in, void *out, const PermParams &pp, int elem_bytes,
                           cudaStream_t s) {
    const int64_t blocks = (int64_t)1 << pp.n_outer;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (pp.tile_bits == 10 && pp.lin == 5 && pp.lout == 5 && pp.n_outer <= 32) {
        const ExpandArgs ex{0, 0, 0};
        if (elem_bytes == 4)
            permute_tiled_kernel<uint32_t, false><<<(unsigned)permute_grid(blocks), 256, 0, s>>>(
                (const uint32_t *)in, out, pp, blocks, ex);
        else if (elem_bytes == 8)
            permute_tiled_kernel<uint2, false><<<(unsigned)permute_grid(blocks), 256, 0, s>>>(
                (const uint2 *)in, out, pp, blocks, ex);
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    const int threads = std::min(256, 1 << pp.tile_bits);
    if (elem_bytes == 4)
        permute_kernel<uint32_t><<<(unsigned)blocks, threads, 0, s>>>(
            (const uint32_t *)in, (uint32_t *)out, pp);
    else if (elem_bytes == 8)
        permute_kernel<uint2><<<(unsigned)blocks, threads, 0, s>>>((const uint2 *)in, (uint2 *)out, pp);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// B (complex-half, any mode order) -> B' in one pass.  `pp` permutes B's
// stored modes into [batch][N][K] order.  Tensors of rank >= 10 with K >= 4
// use the tiled EXPAND kernel; smaller ones a direct gather.
__global__ void bprep_gather_kernel(const uint32_t *__restrict__ B, uint32_t *__restrict__ Bp,
                                    int lk, int ln, int lb, int np, const __grid_constant__ PermParams p,
                                    int rank) {
    const int64_t total = ((int64_t)np << lk) << lb;    // uint32 pairs of B'
    bprep_gather_body(B, Bp, lk, ln, np, p, rank, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, total,
                      (int64_t)gridDim.x * blockDim.x);
}

// B in [batch][N][K] order already: bprep_stream_body, grid-stride
__global__ void __launch_bounds__(256) bprep_stream_kernel(const uint4 *__restrict__ B, uint4 *__restrict__ Bp,
                                                           int lk, int ln, int np, int64_t units) {
    bprep_stream_body<4>(B, Bp, lk, ln, np, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, units,
                         (int64_t)gridDim.x * blockDim.x);
}

// Complex64 B (a small tensor) -> B' in complex-half, one block of 1024
// threads (bprep_c64_body: rounding, 2^s scale, rounding compensation).
template <int DT>
__global__ void __launch_bounds__(1024) bprep_c64_kernel(const float2 *__restrict__ B,
                                                         uint32_t *__restrict__ Bp, int lk, int ln,
                                                         int lb, int np,
                                                         const __grid_constant__ PermParams p,
                                                         int rank, double2 *corr, float *tmax,
                                                         int32_t *texp, int meta_src, int meta_dst,
                                                         int scale_off) {
    __shared__ BprepC64Smem<1024> sm;
    bprep_c64_body<DT, 1024, 1024, SyncBlock>(B, Bp, lk, ln, lb, np, p, rank, corr, tmax, texp, meta_src, meta_dst,
                                              scale_off, threadIdx.x, sm);
}

// The same build over 16 blocks of 64 threads (virtual thread v = one
// thread: the FP64 sums of B's rounding spread over 16 SMs instead of one),
// each virtual thread's sums to part; then one block runs the same tree
// over them (bit-identical to bprep_c64_kernel).
template <int DT>
__global__ void __launch_bounds__(64) bprep_c64_part_kernel(const float2 *__restrict__ B, uint32_t *__restrict__ Bp,
                                                            int lk, int ln, int lb, int np,
                                                            const __grid_constant__ PermParams p, int rank,
                                                            const float *tmax, int meta_src, int scale_off,
                                                            BprepC64Smem<1024> *part) {
    const int v = blockIdx.x * 64 + threadIdx.x;
    const int64_t total = ((int64_t)np << lk) << lb;
    const float scale = __int_as_float((127 + bprep_c64_shift(tmax[meta_src], scale_off)) << 23);
    double nr, ni, den;
    float bmax;
    bprep_c64_vthread<DT, 1024>(B, Bp, lk, ln, np, total, p, rank, scale, v, nr, ni, den, bmax);
    part->sh[0][v] = nr;
    part->sh[1][v] = ni;
    part->sh[2][v] = den;
    part->smax[v] = bmax;
}

__global__ void __launch_bounds__(1024) bprep_c64_reduce_kernel(const BprepC64Smem<1024> *part, double2 *corr,
                                                                float *tmax, int32_t *texp, int meta_src,
                                                                int meta_dst, int scale_off) {
    __shared__ BprepC64Smem<1024> sm;
    const int t = threadIdx.x;
    for (int q = 0; q < 3; ++q) sm.sh[q][t] = part->sh[q][t];
    sm.smax[t] = part->smax[t];
    const int bshift = bprep_c64_shift(tmax[meta_src], scale_off);
    bprep_c64_finish<1024, 1024, SyncBlock>(corr, tmax, texp, meta_src, meta_dst, bshift, t, sm);
}

size_t bprep_c64_scratch_bytes() { return sizeof(BprepC64Smem<1024>); }

cudaError_t launch_bprep_perm(const void *B, void *Bp, int rank, const int32_t *perm, int lk, int ln,
                              int lb, int np, int tb, int dtype, double2 *corr, float *tmax,
                              int32_t *texp, int meta_src, int meta_dst, cudaStream_t s,
                              int scale_off, void *scratch) {
    const ExpandArgs ex{lk, ln, np};
    // direct-gather table: outer_in[t] = input bit position of target bit t
    PermParams g;
    std::memset(&g, 0, sizeof(g));
    for (int i = 0; i < rank; ++i) g.outer_in[rank - 1 - i] = (int8_t)(rank - 1 - perm[i]);
    if (tb == 0 && scratch) {
        auto *part = (BprepC64Smem<1024> *)scratch;
        if (dtype == TN_F16)
            bprep_c64_part_kernel<TN_F16><<<16, 64, 0, s>>>((const float2 *)B, (uint32_t *)Bp, lk, ln, lb, np, g,
                                                            rank, tmax, meta_src, scale_off, part);
        else
            bprep_c64_part_kernel<TN_BF16><<<16, 64, 0, s>>>((const float2 *)B, (uint32_t *)Bp, lk, ln, lb, np, g,
                                                             rank, tmax, meta_src, scale_off, part);
        bprep_c64_reduce_kernel<<<1, 1024, 0, s>>>(part, corr, tmax, texp, meta_src, meta_dst, scale_off);
        return cudaGetLastError();
    }
    if (tb == 0) {
        if (dtype == TN_F16)
            bprep_c64_kernel<TN_F16><<<1, 1024, 0, s>>>((const float2 *)B, (uint32_t *)Bp, lk, ln, lb,
                                                        np, g, rank, corr, tmax, texp, meta_src, meta_dst,
                                                        scale_off);
        else
            bprep_c64_kernel<TN_BF16><<<1, 1024, 0, s>>>((const float2 *)B, (uint32_t *)Bp, lk, ln, lb,
                                                         np, g, rank, corr, tmax, texp, meta_src, meta_dst,
                                                        scale_off);
        return cudaGetLastError();
    }
    bool ident = true;
    for (int i = 0; i < rank; ++i) ident = ident && perm[i] == i;
    if (ident && lk >= 2 && rank == lk + ln + lb && (((uintptr_t)B | (uintptr_t)Bp) & 15) == 0) {
        // 16-byte units: np / 2 row pairs x K / 4 per batch entry
        const int64_t units = ((int64_t)(np >> 1) << (lk - 2)) << lb;
        const int threads = 256;
        const int64_t blocks = std::min<int64_t>((units + threads - 1) / threads, (int64_t)tc_num_sms() * 8);
        bprep_stream_kernel<<<(unsigned)blocks, threads, 0, s>>>((const uint4 *)B, (uint4 *)Bp, lk, ln, np, units);
        return cudaGetLastError();
    }
    if (rank >= 10 && lk >= 2 && np == 2 << ln) {
        const PermParams pp = make_perm_params(rank, perm);
        if (pp.tile_bits == 10 && pp.lin == 5 && pp.lout == 5 && pp.n_outer <= 32) {
            const int64_t blocks = (int64_t)1 << pp.n_outer;
            permute_tiled_kernel<uint32_t, true><<<(unsigned)permute_grid(blocks), 256, 0, s>>>(
                (const uint32_t *)B, Bp, pp, blocks, ex);
            return cudaGetLastError();
        }
    }
    const int64_t total = ((int64_t)np << lk) << lb;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 8192);
    bprep_gather_kernel<<<blocks, threads, 0, s>>>((const uint32_t *)B, (uint32_t *)Bp, lk, ln, lb,
                                                   np, g, rank);
    return cudaGetLastError();
}

// ------------------------------------------- TF32 hi / lo splits (x3) --
// x ~ hi + lo with hi = x rounded to 11 significant bits (TF32: 13 low
// mantissa bits zero, round half away from zero) and lo = x - hi (exact in
// FP32) rounded the same way: both are exactly TF32 values, so the tensor
// cores read them unchanged; |x - hi| <= 2^-11 |x| and lo's own rounding
// <= 2^-23 |x|, and the dropped lo x lo product is <= 2^-22 of |x||y|
__device__ __forceinline__ float round_tf32(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
    hi = round_tf32(x);
    lo = round_tf32(x - hi);
}

__global__ void split_tf32_kernel(const float4 *__restrict__ x, float4 *__restrict__ hi, float4 *__restrict__ lo,
                                  int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = x[i];
        float4 h, l;
        split_tf32(v.x, h.x, l.x);
        split_tf32(v.y, h.y, l.y);
        split_tf32(v.z, h.z, l.z);
        split_tf32(v.w, h.w, l.w);
        hi[i] = h;
        lo[i] = l;
    }
}

cudaError_t launch_split_tf32(const void *x, void *hi, void *lo, int64_t n, cudaStream_t s) {
    if (n % 4 || ((uintptr_t)x | (uintptr_t)hi | (uintptr_t)lo) & 15) return cudaErrorInvalidValue;
    const int64_t n4 = n / 4;
    const int threads = 256;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n4 + threads - 1) / threads, (int64_t)tc_num_sms() * 8));
    split_tf32_kernel<<<(unsigned)blocks, threads, 0, s>>>((const float4 *)x, (float4 *)hi, (float4 *)lo, n4);
    return cudaGetLastError();
}

// complex64 B [batch][K][N] -> the real B' [batch][np][2K] of Eq. 6 in FP32
// as hi and lo parts: row 2n holds (re, -im) and row 2n + 1 (im, re) of
// B[k][n] at columns 2k, 2k + 1; rows 2N .. np - 1 are zero.  One thread per
// (batch entry, B' row, k).
__global__ void bprep_x3_kernel(const float2 *__restrict__ B, float2 *__restrict__ bh, float2 *__restrict__ bl,
                                int lk, int ln, int np, int64_t total) {
    const int K = 1 << lk, N = 1 << ln;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i & (K - 1));
        const int64_t row = i >> lk;
        const int rr = (int)(row % np);
        const int64_t b = row / np;
        const int n = rr >> 1;
        float2 v = make_float2(0.f, 0.f);
        if (n < N) {
            const float2 x = B[((b << lk) + k) * (int64_t)N + n];
            v = (rr & 1) ? make_float2(x.y, x.x) : make_float2(x.x, -x.y);
        }
        float2 h, l;
        split_tf32(v.x, h.x, l.x);
        split_tf32(v.y, h.y, l.y);
        bh[i] = h;
        bl[i] = l;
    }
}

cudaError_t launch_bprep_x3(const void *B, void *bh, void *bl, int lk, int ln, int64_t batch, int np, cudaStream_t s) {
    const int64_t total = (batch * np) << lk;
    const int threads = 256;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads, (int64_t)tc_num_sms() * 8));
    bprep_x3_kernel<<<(unsigned)blocks, threads, 0, s>>>((const float2 *)B, (float2 *)bh, (float2 *)bl, lk, ln, np,
                                                         total);
    return cudaGetLastError();
}

// ----------------------------------------------------------- rows GEMMs --
// Blocks of kRows threads over (row block, column chunk, batch entry):
// rows_body for row blocks blockIdx.x, + gridDim.x, ... < gx and column
// chunks blockIdx.y, + gridDim.y, ... < gy (the grid is capped at a few
// waves and at 65535 chunks; each thread's maximum is recorded once at the
// end).
template <typename TA, typename TB, typename TC, int NC, int DT>
__global__ void __launch_bounds__(kRows) gemm_rows_kernel(
    const TA *__restrict__ A, const TB *__restrict__ B, TC *__restrict__ C, int lm, int ln, int lk,
    int64_t sa, int64_t sb, int64_t sc, ScaleRef sr, const int32_t *za, const int32_t *zb, int64_t gx, int gy) {
    __shared__ RowsSmem<TA, NC> sm;
    float mx = 0.f;
    for (int by = blockIdx.y; by < gy; by += gridDim.y)
        for (int64_t bx = blockIdx.x; bx < gx; bx += gridDim.x)
            rows_body<TA, TB, TC, NC, DT, SyncBlock>(A, B, C, lm, ln, lk, sa, sb, sc, sr, za, zb, bx, by,
                                                     blockIdx.z, threadIdx.x, sm, mx);
    rows_flush<TC, DT>(sr, mx, threadIdx.x);
}

template <typename TA, typename TB, typename TC, int DT>
static cudaError_t rows_dispatch(const void *A, const void *B, void *C, int lm, int ln, int lk,
                                 int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                                 const ScaleRef &sr, cudaStream_t s, const int32_t *za = nullptr,
                                 const int32_t *zb = nullptr) {
    const int64_t M = (int64_t)1 << lm;
    const int N = 1 << ln;
    const int64_t gx = (M + kRows - 1) / kRows;
    if (gx > 0x7fffffffLL || batch > 65535) return cudaErrorInvalidValue;
    // columns per thread: fewer when that is what fills the GPU (a step of
    // few row blocks, e.g. M = 128, N = 128, K = 512, else runs on a handful
    // of SMs); every output's sum is the same whichever thread computes it
    const int64_t fill = 2 * (int64_t)tc_num_sms();
    int ncv = N >= 16 ? 16 : N;
    while (ncv > 1 && gx * ((N + ncv - 1) / ncv) * batch < fill) ncv >>= 1;
    // row blocks per column chunk and batch entry: at most enough for about
    // 8 resident blocks per SM (the rest are looped over)
    const int64_t per = std::max<int64_t>(1, (int64_t)tc_num_sms() * 8 / ((N + ncv - 1) / ncv * batch));
    const int64_t gxl = std::min(gx, per);
#define TN_ROWS_CASE(NCV)                                                                        \
    {                                                                                             \
        const int gy = (N + NCV - 1) / NCV;                                                      \
        dim3 g((unsigned)gxl, (unsigned)std::min(gy, 65535), (unsigned)batch);                   \
        gemm_rows_kernel<TA, TB, TC, NCV, DT><<<g, kRows, 0, s>>>(                                \
            (const TA *)A, (const TB *)B, (TC *)C, lm, ln, lk, sa, sb, sc, sr, za, zb, gx, gy);   \
        break;                                                                                    \
    }
    switch (ncv) {
        case 1: TN_ROWS_CASE(1)
        case 2: TN_ROWS_CASE(2)
        case 4: TN_ROWS_CASE(4)
        case 8: TN_ROWS_CASE(8)
        default: TN_ROWS_CASE(16)
    }
#undef TN_ROWS_CASE
    return cudaGetLastError();
}

cudaError_t launch_gemm_rows_c64(const float2 *A, const float2 *B, float2 *C, int lm, int ln,
                                 int lk, int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                                 cudaStream_t s, const int32_t *za, const int32_t *zb) {
    ScaleRef sr{};
    return rows_dispatch<float2, float2, float2, TN_C64>(A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, za, zb);
}

template <int DT, typename H>
static cudaError_t rows_mixed(int ta, int tb, int tc, const void *A, const void *B, void *C, int lm,
                              int ln, int lk, int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                              const ScaleRef &sr, cudaStream_t s, const int32_t *za, const int32_t *zb) {
    // A is the larger operand, so a complex64 A implies a complex64 B
    const int code = ta * 4 + tb * 2 + tc;
    switch (code) {
        case 0: return rows_dispatch<float2, float2, float2, DT>(A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, za, zb);
        case 1: return rows_dispatch<float2, float2, H, DT>(A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, za, zb);
        case 4: return rows_dispatch<H, float2, float2, DT>(A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, za, zb);
        case 5: return rows_dispatch<H, float2, H, DT>(A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, za, zb);
        case 6: return rows_dispatch<H, H, float2, DT>(A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, za, zb);
        case 7: return rows_dispatch<H, H, H, DT>(A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, za, zb);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gemm_rows_mixed(int dtype, int ta, int tb, int tc, const void *A, const void *B,
                                   void *C, int lm, int ln, int lk, int64_t batch, int64_t sa,
                                   int64_t sb, int64_t sc, const ScaleRef &sr, cudaStream_t s,
                                   const int32_t *za, const int32_t *zb) {
    if (dtype == TN_F16)
        return rows_mixed<TN_F16, __half2>(ta, tb, tc, A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, za, zb);
    return rows_mixed<TN_BF16, __nv_bfloat162>(ta, tb, tc, A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, za,
                                               zb);
}

cudaError_t launch_gemm_rows_lp(int dtype, const void *A, const void *B, void *C, int lm, int ln,
                                int lk, int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                                const ScaleRef &sr, cudaStream_t s) {
    return launch_gemm_rows_mixed(dtype, 1, 1, 1, A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s, nullptr, nullptr);
}

// ---------------------------------------------------------- tiled c64 --
// 64x64 output tile per block of 256 threads (tiled_c64_body).
template <int BM, int BN, int BK, bool LONGK>
__global__ void __launch_bounds__(256) gemm_tiled_c64_kernel(
    const float2 *__restrict__ A, const float2 *__restrict__ B, float2 *__restrict__ C, int lm,
    int ln, int lk, int64_t sa, int64_t sb, int64_t sc, const int32_t *za, const int32_t *zb) {
    __shared__ TiledC64Smem<BM, BN, BK> sm;
    tiled_c64_body<BM, BN, BK, LONGK, SyncBlock>(A, B, C, lm, ln, lk, sa, sb, sc, za, zb, blockIdx.x, blockIdx.y,
                                                 blockIdx.z, threadIdx.x, sm);
}

cudaError_t launch_gemm_tiled_c64(const float2 *A, const float2 *B, float2 *C, int lm, int ln,
                                  int lk, int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                                  int tile, cudaStream_t s, const int32_t *za, const int32_t *zb) {
    (void)tile;
    if (lm < 6 || ln < 6 || lk < 4) return cudaErrorInvalidValue;
    const int64_t gx = ((int64_t)1 << lm) / 64;
    if (gx > 0x7fffffffLL || batch > 65535) return cudaErrorInvalidValue;
    dim3 g((unsigned)gx, (unsigned)((1 << ln) / 64), (unsigned)batch);
    if (lk > 12)
        gemm_tiled_c64_kernel<64, 64, 16, true><<<g, 256, 0, s>>>(A, B, C, lm, ln, lk, sa, sb, sc, za, zb);
    else
        gemm_tiled_c64_kernel<64, 64, 16, false><<<g, 256, 0, s>>>(A, B, C, lm, ln, lk, sa, sb, sc, za, zb);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- bprep --
// B [batch][K][N] complex-half -> B' [batch][np][2K] real (K-major rows):
//   B'[2n  ][2k] =  Re B[k][n],  B'[2n  ][2k+1] = -Im B[k][n]
//   B'[2n+1][2k] =  Im B[k][n],  B'[2n+1][2k+1] =  Re B[k][n]
// rows 2N..np-1 are zero.  (Paper Sec. 3.3, Eq. 6: B padded to
// [B_(real,-imag), B_(imag,real)], the new output mode and the shared
// real/imag mode both innermost.)
template <typename H>
__global__ void bprep_kernel(const H *__restrict__ B, H *__restrict__ Bp, int lk, int ln, int np) {
    const int K = 1 << lk, N = 1 << ln;
    const int64_t per = (int64_t)np * 2 * K;
    const int64_t b = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(i / (2 * K)), col = (int)(i % (2 * K));
        const int n = row >> 1, co = row & 1, k = col >> 1, ci = col & 1;
        H v;
        if (n >= N) {
            v = H(0.0f);
        } else {
            const H *src = B + (b * K + k) * (int64_t)N * 2 + (int64_t)n * 2;
            const H re = src[0], im = src[1];
            if (co == 0) v = ci == 0 ? re : __hneg(im);
            else v = ci == 0 ? im : re;
        }
        Bp[b * per + i] = v;
    }
}

cudaError_t launch_bprep(int dtype, const void *B, void *Bp, int lk, int ln, int64_t batch, int np,
                         cudaStream_t s) {
    const int64_t per = (int64_t)np * 2 * ((int64_t)1 << lk);
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((per + threads - 1) / threads, 4096);
    if (batch > 65535) return cudaErrorInvalidValue;
    dim3 g(blocks, (unsigned)batch);
    if (dtype == TN_F16)
        bprep_kernel<__half><<<g, threads, 0, s>>>((const __half *)B, (__half *)Bp, lk, ln, np);
    else
        bprep_kernel<__nv_bfloat16><<<g, threads, 0, s>>>((const __nv_bfloat16 *)B,
                                                          (__nv_bfloat16 *)Bp, lk, ln, np);
    return cudaGetLastError();
}

// ------------------------------------------------------- E4M3 operands --
template <int DT>
__global__ void quant_e4m3_kernel(const typename LpT<DT>::T2 *__restrict__ src,
                                  __nv_fp8x2_storage_t *__restrict__ dst, int64_t n, float *tmax,
                                  int32_t *texp, int meta_src, int meta_dst) {
    int sh = 0;
    {
        const float m = tmax[meta_src];
        if (m > 0.0f && isfinite(m)) {
            int x;
            frexpf(448.0f / m, &x);           // 2^(x-1) <= 448 / m < 2^x
            sh = max(-120, min(120, x - 1));
        }
    }
    const float sc = exp2i(sh);
    float mx = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = LpT<DT>::to_f2(src[i]);
        v.x *= sc;
        v.y *= sc;
        const __nv_fp8x2_storage_t q = __nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E4M3);
        dst[i] = q;
        const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(q, __NV_E4M3);
        const float2 back = __half22float2(*reinterpret_cast<const __half2 *>(&hr));
        mx = fmaxf(mx, fmaxf(fabsf(back.x), fabsf(back.y)));
    }
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&tmax[meta_dst], mx);
    if (blockIdx.x == 0 && threadIdx.x == 0) texp[meta_dst] = texp[meta_src] + sh;
}

cudaError_t launch_quant_e4m3(const void *src, void *dst, int64_t n_pairs, int dtype, float *tmax,
                              int32_t *texp, int meta_src, int meta_dst, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n_pairs + threads - 1) / threads,
                                                                   (int64_t)tc_num_sms() * 8));
    auto *d = reinterpret_cast<__nv_fp8x2_storage_t *>(dst);
    if (dtype == TN_BF16)
        quant_e4m3_kernel<TN_BF16><<<blocks, threads, 0, s>>>(
            reinterpret_cast<const typename LpT<TN_BF16>::T2 *>(src), d, n_pairs, tmax, texp, meta_src,
            meta_dst);
    else
        quant_e4m3_kernel<TN_F16><<<blocks, threads, 0, s>>>(
            reinterpret_cast<const typename LpT<TN_F16>::T2 *>(src), d, n_pairs, tmax, texp, meta_src,
            meta_dst);
    return cudaGetLastError();
}

// B [batch][K][N] complex E4M3 (re, im bytes) -> B' [batch][np][2K]:
// row (n, 0) = (Re, -Im) per k, row (n, 1) = (Im, Re); E4M3 negation is the
// sign bit.  One uint16 (a k pair) per thread.
__global__ void bprep_e4m3_kernel(const uint16_t *__restrict__ B, uint16_t *__restrict__ Bp, int lk,
                                  int ln, int np) {
    const int K = 1 << lk, N = 1 << ln;
    const int64_t per = (int64_t)np * K;
    const int64_t b = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(i / K), k = (int)(i % K);
        const int n = row >> 1, co = row & 1;
        uint16_t v = 0;
        if (n < N) {
            const uint16_t x = B[(b * K + k) * (int64_t)N + n];
            v = co == 0 ? (uint16_t)(x ^ 0x8000u) : (uint16_t)((x >> 8) | (x << 8));
        }
        Bp[b * per + i] = v;
    }
}

cudaError_t launch_bprep_e4m3(const void *B, void *Bp, int lk, int ln, int64_t batch, int np,
                              cudaStream_t s) {
    const int64_t per = (int64_t)np << lk;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((per + threads - 1) / threads, 4096);
    if (batch > 65535) return cudaErrorInvalidValue;
    dim3 g(blocks, (unsigned)batch);
    bprep_e4m3_kernel<<<g, threads, 0, s>>>((const uint16_t *)B, (uint16_t *)Bp, lk, ln, np);
    return cudaGetLastError();
}

// --------------------------------------------------------- split-K reduce --
template <int DT, bool OUT_C64>
__global__ void splitk_reduce_kernel(const float2 *__restrict__ partial, int split, void *C,
                                     int64_t n, int lk, ScaleRef sr) {
    splitk_body<DT, OUT_C64>(partial, split, C, n, lk, sr, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, n,
                             (int64_t)gridDim.x * blockDim.x, blockIdx.x == 0, threadIdx.x);
}

cudaError_t launch_splitk_reduce(const float *partial, int split, void *C, int out_c64, int dtype,
                                 int64_t batch, int lm, int ln, int lk, const ScaleRef &sr,
                                 cudaStream_t s) {
    const int64_t n = batch << (lm + ln);
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)tc_num_sms() * 8);
    const float2 *p = reinterpret_cast<const float2 *>(partial);
    if (out_c64) {
        if (dtype == TN_F16) splitk_reduce_kernel<TN_F16, true><<<blocks, threads, 0, s>>>(p, split, C, n, lk, sr);
        else splitk_reduce_kernel<TN_BF16, true><<<blocks, threads, 0, s>>>(p, split, C, n, lk, sr);
    } else {
        if (dtype == TN_F16) splitk_reduce_kernel<TN_F16, false><<<blocks, threads, 0, s>>>(p, split, C, n, lk, sr);
        else splitk_reduce_kernel<TN_BF16, false><<<blocks, threads, 0, s>>>(p, split, C, n, lk, sr);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------- slice sum --
// One thread per amplitude (slice_sum_body).
template <typename TF, int DT>
__global__ void slice_sum_kernel(const TF *__restrict__ F, const SumOp op, double2 *amps,
                                 int n_open, int t_lo, int t_hi, int overwrite,
                                 const int32_t *texp, const double2 *__restrict__ stepcorr,
                                 int n_steps, uint64_t split_mask, uint64_t split_val) {
    __shared__ double2 corr;
    if (threadIdx.x == 0) corr = slice_corr(stepcorr, n_steps);
    __syncthreads();
    slice_sum_body<TF, DT>(F, op, amps, n_open, t_lo, t_hi, overwrite, texp, corr, n_steps, split_mask,
                           split_val, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

cudaError_t launch_slice_sum(const void *F, int dtype, const SumOp &op, double2 *amps, int n_open,
                             int t_lo, int t_hi, int overwrite, const int32_t *texp,
                             const double2 *stepcorr, int n_steps, uint64_t split_val, cudaStream_t s) {
    if (op.n_split < 0 || op.n_split > 8 || op.n_split > n_open) return cudaErrorInvalidValue;
    uint64_t split_mask = 0;
    for (int i = 0; i < op.n_split; ++i) split_mask |= 1ull << op.split_t[i];
    if ((split_val & ~split_mask) != 0) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)1 << (n_open - op.n_split);
    // one thread per amplitude, each summing every slice in FP64: blocks of
    // as few as 32 threads so that the FP64 work spreads over the SMs
    int threads = 32;
    while (threads < 256 && n / (2 * threads) >= tc_num_sms()) threads *= 2;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    if (dtype == TN_C64)
        slice_sum_kernel<float2, TN_C64><<<blocks, threads, 0, s>>>(
            (const float2 *)F, op, amps, n_open, t_lo, t_hi, overwrite, nullptr, nullptr, 0, split_mask, split_val);
    else if (op.tf == 0 && dtype == TN_F16)
        slice_sum_kernel<float2, TN_F16><<<blocks, threads, 0, s>>>(
            (const float2 *)F, op, amps, n_open, t_lo, t_hi, overwrite, texp, stepcorr, n_steps, split_mask, split_val);
    else if (op.tf == 0)
        slice_sum_kernel<float2, TN_BF16><<<blocks, threads, 0, s>>>(
            (const float2 *)F, op, amps, n_open, t_lo, t_hi, overwrite, texp, stepcorr, n_steps, split_mask, split_val);
    else if (dtype == TN_F16)
        slice_sum_kernel<__half2, TN_F16><<<blocks, threads, 0, s>>>(
            (const __half2 *)F, op, amps, n_open, t_lo, t_hi, overwrite, texp, stepcorr, n_steps, split_mask, split_val);
    else
        slice_sum_kernel<__nv_bfloat162, TN_BF16><<<blocks, threads, 0, s>>>(
            (const __nv_bfloat162 *)F, op, amps, n_open, t_lo, t_hi, overwrite, texp, stepcorr,
            n_steps, split_mask, split_val);
    return cudaGetLastError();
}

// --------------------------------------------------------------- metrics --
// FP64 reductions, deterministic: each block sums a fixed strided subset in
// a fixed tree order into partials[block][5]; one block then adds the
// partials in block order.  Sums: |r|^2, |b|^2, |r-b|^2, Re<b,r>, Im<b,r>.
__device__ __forceinline__ void block_sum5(double v[5], double *sh /* [5][256] */) {
    for (int q = 0; q < 5; ++q) sh[q * 256 + threadIdx.x] = v[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 5; ++q) sh[q * 256 + threadIdx.x] += sh[q * 256 + threadIdx.x + w];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) metrics_partial_kernel(const double2 *r, const double2 *b,
                                                              int64_t n, double *partials) {
    __shared__ double sh[5 * 256];
    double v[5] = {0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const double2 x = r[i];
        v[0] += x.x * x.x + x.y * x.y;
        if (b) {
            const double2 y = b[i];
            v[1] += y.x * y.x + y.y * y.y;
            const double dx = x.x - y.x, dy = x.y - y.y;
            v[2] += dx * dx + dy * dy;
            v[3] += y.x * x.x + y.y * x.y;   // Re conj(b) r
            v[4] += y.x * x.y - y.y * x.x;   // Im conj(b) r
        }
    }
    block_sum5(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) partials[(int64_t)blockIdx.x * 5 + q] = sh[q * 256];
}

__global__ void __launch_bounds__(256) metrics_final_kernel(const double *partials, int n_blocks,
                                                            double *out5) {
    __shared__ double sh[5 * 256];
    double v[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n_blocks; i += 256)
        for (int q = 0; q < 5; ++q) v[q] += partials[(int64_t)i * 5 + q];
    block_sum5(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) out5[q] = sh[q * 256];
}

cudaError_t launch_metrics(const double2 *r, const double2 *b, int64_t n, double *d_out5,
                           double *d_partials, int n_blocks, cudaStream_t s) {
    metrics_partial_kernel<<<n_blocks, 256, 0, s>>>(r, b, n, d_partials);
    metrics_final_kernel<<<1, 256, 0, s>>>(d_partials, n_blocks, d_out5);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ top-k --
// Post-selection: k rounds; round i finds the first element, in the total
// order (p descending, index ascending), that comes after the element
// chosen in round i-1.  One block; p = |amp|^2 in FP64.
__device__ __forceinline__ bool before(double p1, int64_t i1, double p2, int64_t i2) {
    return p1 > p2 || (p1 == p2 && i1 < i2);
}

__global__ void __launch_bounds__(1024) topk_kernel(const double2 *amps, int64_t n, int k,
                                                    int64_t *out_idx, double *out_prob) {
    __shared__ double sp[1024];
    __shared__ int64_t si[1024];
    double prev_p = INFINITY;
    int64_t prev_i = -1;
    for (int round = 0; round < k; ++round) {
        double bp = -1.0;
        int64_t bi = -1;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const double2 a = amps[i];
            // |a|^2 with each product and the sum rounded once (no FMA), so the
            // selection matches any other FP64 evaluation of re*re + im*im
            const double p = __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
            if (!before(p, i, prev_p, prev_i) && !(p == prev_p && i == prev_i)) {
                if (bi < 0 || before(p, i, bp, bi)) { bp = p; bi = i; }
            }
        }
        sp[threadIdx.x] = bp;
        si[threadIdx.x] = bi;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) {
                const double p2 = sp[threadIdx.x + w];
                const int64_t i2 = si[threadIdx.x + w];
                if (i2 >= 0 && (si[threadIdx.x] < 0 || before(p2, i2, sp[threadIdx.x], si[threadIdx.x]))) {
                    sp[threadIdx.x] = p2;
                    si[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        prev_p = sp[0];
        prev_i = si[0];
        if (threadIdx.x == 0) {
            out_idx[round] = prev_i;
            out_prob[round] = prev_p;
        }
        __syncthreads();
    }
}

cudaError_t launch_topk(const double2 *amps, int64_t n, int k, int64_t *d_idx, double *d_prob,
                        cudaStream_t s) {
    topk_kernel<<<1, 1024, 0, s>>>(amps, n, k, d_idx, d_prob);
    return cudaGetLastError();
}

// Top-k over many blocks, O(n) reads per pass: the same total order (p
// descending, index ascending; p = re*re + im*im rounded as above).  p >= 0,
// so the bits of p, read as an unsigned 64-bit integer, order like p.
//  1. radix select, 8 passes of 8 bits from the top: each pass histograms
//     the next byte of the keys that match the bytes fixed so far, and one
//     thread fixes the byte at which the count from the top reaches the
//     number still wanted -- after 8 passes the k-th largest key T is known,
//     and kk, how many of the keys equal to T belong to the top k;
//  2. every key above T is kept, and of the keys equal to T the kk with the
//     lowest indices (per-block counts, an exclusive scan over the blocks,
//     and a block-wide scan in index order inside each block);
//  3. the k kept entries are sorted by the total order (bitonic: in shared
//     memory up to 2048 entries, else over global memory).
struct TopkHead {
    uint64_t prefix, mask;
    int64_t kk;            // keys equal to the threshold that are kept
    int64_t n_gt;          // keys above the threshold (k - kk at the end)
    uint32_t gt_pos;       // write cursor of the keys above the threshold
    uint32_t pad_;
    uint32_t hist[256];
};
constexpr int kTopkMaxBlocks = 1024;
constexpr int kTopkSmallSort = 2048;

__device__ __forceinline__ uint64_t topk_key(double2 a) {
    return (uint64_t)__double_as_longlong(__dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)));
}

__global__ void topk_init_kernel(TopkHead *h, int64_t k) {
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h->hist[t] = 0u;
    if (threadIdx.x == 0) {
        h->prefix = 0;
        h->mask = 0;
        h->kk = k;
        h->n_gt = 0;
        h->gt_pos = 0;
    }
}

__global__ void __launch_bounds__(256) topk_hist_kernel(const double2 *amps, int64_t n, TopkHead *h, int shift) {
    __shared__ uint32_t sh[256];
    sh[threadIdx.x] = 0u;
    __syncthreads();
    const uint64_t prefix = h->prefix, mask = h->mask;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = topk_key(amps[i]);
        if ((key & mask) == prefix) atomicAdd(&sh[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (sh[threadIdx.x]) atomicAdd(&h->hist[threadIdx.x], sh[threadIdx.x]);
}

__global__ void topk_select_kernel(TopkHead *h, int shift) {
    if (threadIdx.x != 0) return;
    int64_t need = h->kk, cum = 0;
    int digit = 0;
    for (int v = 255; v >= 0; --v) {
        const int64_t c = h->hist[v];
        if (cum + c >= need) {
            digit = v;
            break;
        }
        cum += c;
    }
    h->prefix |= (uint64_t)digit << shift;
    h->mask |= (uint64_t)0xFF << shift;
    h->kk = need - cum;
    for (int t = 0; t < 256; ++t) h->hist[t] = 0u;
}

__global__ void __launch_bounds__(256) topk_count_kernel(const double2 *amps, int64_t n, const TopkHead *h,
                                                         int64_t chunk, int64_t *blockcnt) {
    __shared__ int64_t sw[8];
    const uint64_t T = h->prefix;
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    int64_t c = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) c += topk_key(amps[i]) == T;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < 8; ++w) t += sw[w];
        blockcnt[blockIdx.x] = t;
    }
}

__global__ void topk_offsets_kernel(int64_t *blockcnt, int nblk, TopkHead *h, int64_t k) {
    if (threadIdx.x != 0) return;
    int64_t run = 0;
    for (int b = 0; b < nblk; ++b) {
        const int64_t c = blockcnt[b];
        blockcnt[b] = run;
        run += c;
    }
    h->n_gt = k - h->kk;
    h->gt_pos = 0;
}

__global__ void __launch_bounds__(256) topk_collect_kernel(const double2 *amps, int64_t n, TopkHead *h,
                                                           int64_t chunk, const int64_t *offsets, int64_t *cand_idx,
                                                           double *cand_p) {
    __shared__ int s_warp[8];
    const uint64_t T = h->prefix;
    const int64_t kk = h->kk, n_gt = h->n_gt;
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t run = offsets[blockIdx.x];      // rank of the next equal key in index order
    for (int64_t base = i0; base < i1; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        uint64_t key = 0;
        double p = 0.0;
        const bool valid = i < i1;
        if (valid) {
            const double2 a = amps[i];
            p = __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
            key = (uint64_t)__double_as_longlong(p);
        }
        if (valid && key > T) {
            const uint32_t pos = atomicAdd(&h->gt_pos, 1u);
            cand_idx[pos] = i;
            cand_p[pos] = p;
        }
        const bool eq = valid && key == T;
        const uint32_t bal = __ballot_sync(0xffffffffu, eq);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        int64_t before = 0, total = 0;
        for (int w = 0; w < 8; ++w) {
            if (w < warp) before += s_warp[w];
            total += s_warp[w];
        }
        if (eq) {
            const int64_t rank = run + before + __popc(bal & ((1u << lane) - 1u));
            if (rank < kk) {
                cand_idx[n_gt + rank] = i;
                cand_p[n_gt + rank] = p;
            }
        }
        run += total;
        __syncthreads();
    }
}

__device__ __forceinline__ void topk_cmpswap(int64_t &ia, double &pa, int64_t &ib, double &pb, bool up) {
    // up: a must come before b in the total order
    const bool b_first = before(pb, ib, pa, ia);
    if (b_first == up) {
        const int64_t ti = ia;
        ia = ib;
        ib = ti;
        const double tp = pa;
        pa = pb;
        pb = tp;
    }
}

__global__ void __launch_bounds__(1024) topk_sort_small_kernel(const int64_t *cand_idx, const double *cand_p, int k,
                                                               int P, int64_t *out_idx, double *out_prob) {
    __shared__ int64_t si[kTopkSmallSort];
    __shared__ double sp[kTopkSmallSort];
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        si[t] = t < k ? cand_idx[t] : INT64_MAX;
        sp[t] = t < k ? cand_p[t] : -1.0;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1)), j = i + stride;
                topk_cmpswap(si[i], sp[i], si[j], sp[j], (i & size) == 0);
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        out_idx[t] = si[t];
        out_prob[t] = sp[t];
    }
}

__global__ void topk_pad_kernel(int64_t *cand_idx, double *cand_p, int64_t k, int64_t P) {
    for (int64_t t = k + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x) {
        cand_idx[t] = INT64_MAX;
        cand_p[t] = -1.0;
    }
}

__global__ void topk_bitonic_kernel(int64_t *cand_idx, double *cand_p, int64_t P, int64_t size, int64_t stride) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P / 2; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = 2 * t - (t & (stride - 1)), j = i + stride;
        int64_t ia = cand_idx[i], ib = cand_idx[j];
        double pa = cand_p[i], pb = cand_p[j];
        topk_cmpswap(ia, pa, ib, pb, (i & size) == 0);
        cand_idx[i] = ia;
        cand_idx[j] = ib;
        cand_p[i] = pa;
        cand_p[j] = pb;
    }
}

__global__ void topk_copy_kernel(const int64_t *cand_idx, const double *cand_p, int64_t k, int64_t *out_idx,
                                 double *out_prob) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k; t += (int64_t)gridDim.x * blockDim.x) {
        out_idx[t] = cand_idx[t];
        out_prob[t] = cand_p[t];
    }
}

static int64_t topk_pad(int64_t k) {
    int64_t P = 1;
    while (P < k) P <<= 1;
    return P;
}

bool topk_one_block(int64_t n, int64_t k) { return k * n <= ((int64_t)1 << 22); }

size_t topk_scratch_bytes(int64_t n, int64_t k) {
    if (topk_one_block(n, k)) return 0;
    const int64_t P = k <= kTopkSmallSort ? k : topk_pad(k);
    return 4096 + (size_t)kTopkMaxBlocks * 8 + (size_t)P * 16;
}

cudaError_t launch_topk_select(const double2 *amps, int64_t n, int64_t k, void *scratch, int64_t *d_idx,
                               double *d_prob, cudaStream_t s) {
    if (k < 1 || k > n) return cudaErrorInvalidValue;
    if (topk_one_block(n, k)) return launch_topk(amps, n, (int)k, d_idx, d_prob, s);
    if (!scratch) return cudaErrorInvalidValue;
    const int64_t P = k <= kTopkSmallSort ? k : topk_pad(k);
    char *base = (char *)scratch;
    TopkHead *h = (TopkHead *)base;
    int64_t *blockcnt = (int64_t *)(base + 4096);
    int64_t *cand_idx = (int64_t *)(base + 4096 + (size_t)kTopkMaxBlocks * 8);
    double *cand_p = (double *)(cand_idx + P);
    topk_init_kernel<<<1, 256, 0, s>>>(h, k);
    const int hist_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 2047) / 2048, (int64_t)tc_num_sms() * 4));
    for (int shift = 56; shift >= 0; shift -= 8) {
        topk_hist_kernel<<<hist_blocks, 256, 0, s>>>(amps, n, h, shift);
        topk_select_kernel<<<1, 32, 0, s>>>(h, shift);
    }
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(kTopkMaxBlocks, (n + 4095) / 4096));
    const int64_t chunk = (n + nblk - 1) / nblk;
    topk_count_kernel<<<nblk, 256, 0, s>>>(amps, n, h, chunk, blockcnt);
    topk_offsets_kernel<<<1, 32, 0, s>>>(blockcnt, nblk, h, k);
    topk_collect_kernel<<<nblk, 256, 0, s>>>(amps, n, h, chunk, blockcnt, cand_idx, cand_p);
    if (k <= kTopkSmallSort) {
        int P2 = 1;
        while (P2 < k) P2 <<= 1;
        topk_sort_small_kernel<<<1, 1024, 0, s>>>(cand_idx, cand_p, (int)k, P2, d_idx, d_prob);
        return cudaGetLastError();
    }
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((P / 2 + 255) / 256, (int64_t)tc_num_sms() * 8));
    topk_pad_kernel<<<blocks, 256, 0, s>>>(cand_idx, cand_p, k, P);
    for (int64_t size = 2; size <= P; size <<= 1)
        for (int64_t stride = size >> 1; stride > 0; stride >>= 1)
            topk_bitonic_kernel<<<blocks, 256, 0, s>>>(cand_idx, cand_p, P, size, stride);
    topk_copy_kernel<<<blocks, 256, 0, s>>>(cand_idx, cand_p, k, d_idx, d_prob);
    return cudaGetLastError();
}

}  // namespace tn
