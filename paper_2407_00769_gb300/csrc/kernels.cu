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

#include "kernels.cuh"

namespace tn {

// ------------------------------------------------------------ lp helpers --
template <int DT> struct LpT;
template <> struct LpT<TN_F16> {
    using T2 = __half2;
    static __device__ __forceinline__ float2 to_f2(T2 v) { return __half22float2(v); }
    static __device__ __forceinline__ T2 from_f2(float2 v) { return __floats2half2_rn(v.x, v.y); }
    static __device__ __forceinline__ T2 from_d2(double re, double im) {
        return __halves2half2(__double2half(re), __double2half(im));
    }
};
template <> struct LpT<TN_BF16> {
    using T2 = __nv_bfloat162;
    static __device__ __forceinline__ float2 to_f2(T2 v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ T2 from_f2(float2 v) { return __floats2bfloat162_rn(v.x, v.y); }
    static __device__ __forceinline__ T2 from_d2(double re, double im) {
        return __halves2bfloat162(__double2bfloat16(re), __double2bfloat16(im));
    }
};

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ void atomic_max_nonneg(float *addr, float v) {
    atomicMax(reinterpret_cast<int *>(addr), __float_as_int(v));
}

// exponent e for a product of two scaled tensors: with |A| <= sqrt2 maxA,
// |B| <= sqrt2 maxB and K terms, |C| <= 2 K maxA maxB; choose e so that
// 2 K maxA maxB 2^e <= 2^14 (FP16 max is 65504 ~ 2^16).
__device__ __forceinline__ int scale_exponent(float maxa, float maxb, int lk) {
    const float t = 2.0f * maxa * maxb;
    if (!(t > 0.0f) || !isfinite(t)) return 0;
    int x;
    const float f = frexpf(t, &x);            // t = f 2^x, f in [0.5, 1)
    const int c = (f == 0.5f) ? x - 1 : x;    // ceil(log2 t)
    int e = 14 - lk - c;
    return max(-120, min(120, e));
}

__device__ __forceinline__ float exp2i(int e) {   // exact 2^e, |e| <= 126
    return __int_as_float((127 + e) << 23);
}

// ------------------------------------------------------------- leaf prep --
// One block per leaf.  Output element o (over the kept legs) reads input
// element in(o) = kept bits placed at keep_pos, fixed legs at the value of
// their slice-id bit (slice decoding: bit j of the slice id is sliced edge
// j's value).  Converts complex128 -> the contraction dtype (RN).
__global__ void leaf_prep_kernel(const LeafJob *jobs, const double2 *store, char *ws,
                                 int64_t slice_base, float *tmax, int32_t *texp) {
    const LeafJob j = jobs[blockIdx.x];
    const int n_out = 1 << j.rank_out;
    float m = 0.0f;
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
        int64_t in = 0;
        for (int i = 0; i < j.rank_out; ++i)
            if ((o >> i) & 1) in |= (int64_t)1 << j.keep_pos[i];
        for (int f = 0; f < j.n_fixed; ++f)
            in |= ((slice_base >> j.fixed_bit[f]) & 1) << j.fixed_pos[f];
        const double2 v = store[j.src + in];
        const float2 w = make_float2((float)v.x, (float)v.y);
        reinterpret_cast<float2 *>(ws + j.dst)[o] = w;
        m = fmaxf(m, fmaxf(fabsf(w.x), fabsf(w.y)));
    }
    if (tmax) {
        m = warp_max(m);
        __shared__ float sm[32];
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            float mm = 0.0f;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) mm = fmaxf(mm, sm[w]);
            tmax[j.meta] = mm;
            texp[j.meta] = 0;
        }
    }
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
    int64_t bin = 0, bout = 0;
    const int64_t tid = blockIdx.x;
    for (int k = 0; k < p.n_outer; ++k)
        if ((tid >> k) & 1) {
            bin |= (int64_t)1 << p.outer_in[k];
            bout |= (int64_t)1 << p.outer_out[k];
        }
    const int n = 1 << p.tile_bits;
    const int lo_mask_in = (1 << p.lin) - 1;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int64_t off = bin + (e & lo_mask_in) + p.rd_hi_off[e >> p.lin];
        tile[e + (e >> 5)] = in[off];
    }
    __syncthreads();
    const int lo_mask_out = (1 << p.lout) - 1;
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
        const int fl = f & lo_mask_out, fh = f >> p.lout;
        const int e = p.wr_lo_e[fl] | p.wr_hi_e[fh];
        out[bout + fl + p.wr_hi_off[fh]] = tile[e + (e >> 5)];
    }
}

// Fast path for tensors of rank >= 10: the tile is always 2^10 elements
// (32 contiguous input elements x 32 contiguous output elements), and the
// position of an element inside its tile is the same for every tile, so
// each thread works out once where its 4 elements come from and go to; per
// tile only the tile's base offsets change (from 8-bit lookup tables).  Each
// thread moves its 4 elements with one 16-byte (4-byte elements) or two
// (8-byte elements) vector loads and stores.  Persistent over tiles.
//
// EXPAND (complex-half only): instead of the permuted tensor, write the
// padded real operand of the tensor-core GEMM (Sec. 3.3, Eq. 6): the
// permuted order is [batch][N][K] complex and element (b, n, k) = (re, im)
// goes to B'[b][2n][k] = (re, -im) and B'[b][2n+1][k] = (im, re) (pairs of
// halves; np rows per batch).
struct ExpandArgs {
    int32_t lk, ln, np;
};

template <typename T, bool EXPAND>
__global__ void __launch_bounds__(256) permute_tiled_kernel(const T *__restrict__ in,
                                                            void *__restrict__ out_,
                                                            const __grid_constant__ PermParams p,
                                                            int64_t ntiles, ExpandArgs ex) {
    __shared__ T tile[2][1024 + 32];
    __shared__ int64_t s_bin[4][256], s_bout[4][256];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        const int level = i >> 8, v = i & 255;
        int64_t bi = 0, bo = 0;
        for (int b = 0; b < 8; ++b) {
            const int k = level * 8 + b;
            if (k < p.n_outer && ((v >> b) & 1)) {
                bi |= (int64_t)1 << p.outer_in[k];
                bo |= (int64_t)1 << p.outer_out[k];
            }
        }
        s_bin[level][v] = bi;
        s_bout[level][v] = bo;
    }
    // this thread's 4 elements: read-order e0..e0+3, write-order f0..f0+3
    const int e0 = threadIdx.x * 4;
    const int64_t in_off = (e0 & 31) + p.rd_hi_off[e0 >> 5];
    int rd_slot[4], wr_slot[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        rd_slot[j] = (e0 + j) + ((e0 + j) >> 5);
        const int f = e0 + j;
        const int e = p.wr_lo_e[f & 31] | p.wr_hi_e[f >> 5];
        wr_slot[j] = e + (e >> 5);
    }
    const int64_t out_off = (e0 & 31) + p.wr_hi_off[e0 >> 5];
    __syncthreads();
    // two tiles per iteration (two 16-byte loads in flight per thread)
    for (int64_t t0 = blockIdx.x; t0 < ntiles; t0 += 2 * (int64_t)gridDim.x) {
        const int64_t t1 = t0 + gridDim.x;
        const bool has1 = t1 < ntiles;
        T v[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t t = h ? t1 : t0;
            if (h && !has1) break;
            const int64_t bin = s_bin[0][t & 255] + s_bin[1][(t >> 8) & 255] +
                                s_bin[2][(t >> 16) & 255] + s_bin[3][(t >> 24) & 255];
            if constexpr (sizeof(T) == 4) {
                const uint4 x = *reinterpret_cast<const uint4 *>(in + bin + in_off);
                v[h][0] = x.x; v[h][1] = x.y; v[h][2] = x.z; v[h][3] = x.w;
            } else {
                const uint4 x = *reinterpret_cast<const uint4 *>(in + bin + in_off);
                const uint4 y = *reinterpret_cast<const uint4 *>(in + bin + in_off + 2);
                v[h][0] = make_uint2(x.x, x.y); v[h][1] = make_uint2(x.z, x.w);
                v[h][2] = make_uint2(y.x, y.y); v[h][3] = make_uint2(y.z, y.w);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h && !has1) break;
#pragma unroll
            for (int j = 0; j < 4; ++j) tile[h][rd_slot[j]] = v[h][j];
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t t = h ? t1 : t0;
            if (h && !has1) break;
            const int64_t bout = s_bout[0][t & 255] + s_bout[1][(t >> 8) & 255] +
                                 s_bout[2][(t >> 16) & 255] + s_bout[3][(t >> 24) & 255];
            T w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = tile[h][wr_slot[j]];
            const int64_t f = bout + out_off;
            if constexpr (EXPAND) {
                const int K = 1 << ex.lk;
                const int64_t k0 = f & (K - 1);
                const int64_t n = (f >> ex.lk) & ((1 << ex.ln) - 1);
                const int64_t b = f >> (ex.lk + ex.ln);
                uint32_t *o = reinterpret_cast<uint32_t *>(out_);
                const int64_t row0 = b * ex.np + 2 * n;
                uint4 r0, r1;
                // (re, -im): flip the sign bit of the high half; (im, re): swap halves
                r0.x = w[0] ^ 0x80000000u; r0.y = w[1] ^ 0x80000000u;
                r0.z = w[2] ^ 0x80000000u; r0.w = w[3] ^ 0x80000000u;
                r1.x = __byte_perm(w[0], 0, 0x1032); r1.y = __byte_perm(w[1], 0, 0x1032);
                r1.z = __byte_perm(w[2], 0, 0x1032); r1.w = __byte_perm(w[3], 0, 0x1032);
                *reinterpret_cast<uint4 *>(o + row0 * K + k0) = r0;
                *reinterpret_cast<uint4 *>(o + (row0 + 1) * K + k0) = r1;
            } else {
                T *out = reinterpret_cast<T *>(out_);
                if constexpr (sizeof(T) == 4) {
                    *reinterpret_cast<uint4 *>(out + f) = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
                    *reinterpret_cast<uint4 *>(out + f) = make_uint4(w[0].x, w[0].y, w[1].x, w[1].y);
                    *reinterpret_cast<uint4 *>(out + f + 2) = make_uint4(w[2].x, w[2].y, w[3].x, w[3].y);
                }
            }
        }
        __syncthreads();
    }
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
    // target complex index bits: [batch][N][K], LSB = k bit 0.  For target
    // bit i the input bit position is in_pos = r-1-perm[r-1-i].
    const int K = 1 << lk, N = 1 << ln;
    const int64_t total = ((int64_t)np * K) << lb;    // uint32 pairs of B'
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % K);
        const int64_t row = i / K;
        const int rr = (int)(row % np);
        const int64_t b = row / np;
        const int n = rr >> 1, co = rr & 1;
        uint32_t v = 0;
        if (n < N) {
            const int64_t tidx = ((b * N + n) << lk) | k;
            int64_t src = 0;
            for (int t = 0; t < rank; ++t)
                if ((tidx >> t) & 1) src |= (int64_t)1 << p.outer_in[t];
            const uint32_t x = B[src];
            v = co == 0 ? (x ^ 0x80000000u) : __byte_perm(x, 0, 0x1032);
        }
        Bp[i] = v;
    }
}

// Complex64 B (a small tensor) -> B' in complex-half, one block: every
// element is rounded to the plan's dtype here, and the rounding's component
// along B, alpha = <B, B~ - B> / <B, B>, is measured (FP64, fixed order) so
// the final sum can divide the factor (1 + alpha) out exactly (the network is
// linear in B): corr = 1 / (1 + alpha).
template <int DT>
__global__ void __launch_bounds__(1024) bprep_c64_kernel(const float2 *__restrict__ B,
                                                         uint32_t *__restrict__ Bp, int lk, int ln,
                                                         int lb, int np,
                                                         const __grid_constant__ PermParams p,
                                                         int rank, double2 *corr, float *tmax,
                                                         int32_t *texp, int meta_src, int meta_dst,
                                                         int scale_off) {
    using L = LpT<DT>;
    const int K = 1 << lk, N = 1 << ln;
    const int64_t total = ((int64_t)np * K) << lb;
    // exact power-of-two scale bringing max |B| to [2^11, 2^12]
    int bshift = 0;
    {
        const float mb = tmax[meta_src];
        if (!scale_off && mb > 0.0f && isfinite(mb)) {
            int x;
            const float f = frexpf(mb, &x);
            bshift = 12 - ((f == 0.5f) ? x - 1 : x);
            bshift = max(-120, min(120, bshift));
        }
    }
    const float scale = __int_as_float((127 + bshift) << 23);
    float bmax = 0.0f;
    double nr = 0.0, ni = 0.0, den = 0.0;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const int k = (int)(i % K);
        const int64_t row = i / K;
        const int rr = (int)(row % np);
        const int64_t b = row / np;
        const int n = rr >> 1, co = rr & 1;
        uint32_t v = 0;
        if (n < N) {
            const int64_t tidx = ((b * N + n) << lk) | k;
            int64_t src = 0;
            for (int t = 0; t < rank; ++t)
                if ((tidx >> t) & 1) src |= (int64_t)1 << p.outer_in[t];
            const float2 x0 = B[src];
            const float2 x = make_float2(x0.x * scale, x0.y * scale);
            const typename L::T2 h = L::from_f2(x);
            const uint32_t u = *reinterpret_cast<const uint32_t *>(&h);
            v = co == 0 ? (u ^ 0x80000000u) : __byte_perm(u, 0, 0x1032);
            if (co == 0) {
                const float2 r = L::to_f2(h);
                bmax = fmaxf(bmax, fmaxf(fabsf(r.x), fabsf(r.y)));
                const double dr = (double)r.x - x.x, di = (double)r.y - x.y;
                nr += (double)x.x * dr + (double)x.y * di;     // Re conj(x) d
                ni += (double)x.x * di - (double)x.y * dr;     // Im conj(x) d
                den += (double)x.x * x.x + (double)x.y * x.y;
            }
        }
        Bp[i] = v;
    }
    __shared__ double sh[3][1024];
    __shared__ float smax[1024];
    sh[0][threadIdx.x] = nr;
    sh[1][threadIdx.x] = ni;
    sh[2][threadIdx.x] = den;
    smax[threadIdx.x] = bmax;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
            smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tmax[meta_dst] = smax[0];
        texp[meta_dst] = texp[meta_src] + bshift;
    }
    if (threadIdx.x == 0 && corr) {
        double fr = 1.0, fi = 0.0;
        if (sh[2][0] > 0.0) {
            // 1 / (1 + alpha)
            const double ar = 1.0 + sh[0][0] / sh[2][0], ai = sh[1][0] / sh[2][0];
            const double d = ar * ar + ai * ai;
            fr = ar / d;
            fi = -ai / d;
        }
        *corr = make_double2(fr, fi);
    }
}

cudaError_t launch_bprep_perm(const void *B, void *Bp, int rank, const int32_t *perm, int lk, int ln,
                              int lb, int np, int tb, int dtype, double2 *corr, float *tmax,
                              int32_t *texp, int meta_src, int meta_dst, cudaStream_t s,
                              int scale_off) {
    const ExpandArgs ex{lk, ln, np};
    // direct-gather table: outer_in[t] = input bit position of target bit t
    PermParams g;
    std::memset(&g, 0, sizeof(g));
    for (int i = 0; i < rank; ++i) g.outer_in[rank - 1 - i] = (int8_t)(rank - 1 - perm[i]);
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

// ----------------------------------------------------------- rows GEMMs --
// C[b][m][n] = sum_k A[b][m][k] B[b][k][n].  A block owns ROWS consecutive
// rows (one per thread) and NC consecutive columns (grid.y); the A tile is
// staged through shared memory with coalesced 16-byte loads (its rows are
// contiguous), B's column chunk sits in shared memory as FP32 complex.
// K is walked in chunks of KC.
constexpr int kRows = 128;
constexpr int kKC = 32;
constexpr int kFlushK = 256;   // FP32 terms per partial sum before the FP64 add

// operand conversion: complex64 as is, complex-half widened to FP32
template <typename T, int DT>
__device__ __forceinline__ float2 widen(T v) {
    if constexpr (std::is_same<T, float2>::value) return v;
    else return LpT<DT>::to_f2(v);
}

// Operand and result storage may differ (complex-half plans keep small
// tensors in complex64): TA, TB, TC are float2 or the plan's complex-half
// type, DT the plan's dtype.
template <typename TA, typename TB, typename TC, int NC, int DT>
__global__ void __launch_bounds__(kRows) gemm_rows_kernel(
    const TA *__restrict__ A, const TB *__restrict__ B, TC *__restrict__ C, int lm, int ln, int lk,
    int64_t sa, int64_t sb, int64_t sc, ScaleRef sr, const int32_t *za, const int32_t *zb) {
    constexpr int KC = kKC;
    __shared__ __align__(16) TA As[kRows * KC];
    __shared__ float2 Bs[KC][NC];
    const int64_t M = (int64_t)1 << lm;
    const int N = 1 << ln, K = 1 << lk;
    const int64_t b = blockIdx.z;
    const int64_t m0 = (int64_t)blockIdx.x * kRows;
    const int n0 = blockIdx.y * NC;
    const int nc = min(NC, N);
    // sparse-state gathers: operand chunks by index instead of by batch entry
    const TA *Ab = A + (za ? (int64_t)za[b] : b) * sa;
    const TB *Bb = B + (zb ? (int64_t)zb[b] : b) * sb;
    TC *Cb = C + b * sc;
    const int rows = (int)min((int64_t)kRows, M - m0);
    // FP32 partial sums over at most kFlushK terms, added into FP64: a long
    // FP32 running sum would lose ~sqrt(K) ulps (2^23-term steps occur)
    float2 acc[NC];
    double2 tot[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        acc[j] = make_float2(0.f, 0.f);
        tot[j] = make_double2(0.0, 0.0);
    }
    for (int k0 = 0; k0 < K; k0 += KC) {
        const int kc = min(KC, K - k0);
        __syncthreads();
        // A tile: rows x kc elements; when kc == K the tile is contiguous
        {
            const int per16 = 16 / (int)sizeof(TA);
            const int total = rows * kc;
            if (kc == K && (total % per16) == 0) {
                const uint4 *src = reinterpret_cast<const uint4 *>(Ab + m0 * K);
                uint4 *dst = reinterpret_cast<uint4 *>(As);
                for (int i = threadIdx.x; i < total / per16; i += kRows) dst[i] = src[i];
            } else {
                for (int i = threadIdx.x; i < total; i += kRows) {
                    const int r = i / kc, kk = i % kc;
                    As[r * kc + kk] = Ab[(m0 + r) * K + k0 + kk];
                }
            }
        }
        for (int i = threadIdx.x; i < kc * nc; i += kRows) {
            const int kk = i / nc, j = i % nc;
            Bs[kk][j] = widen<TB, DT>(Bb[(int64_t)(k0 + kk) * N + n0 + j]);
        }
        __syncthreads();
        if (threadIdx.x < rows) {
            for (int kk = 0; kk < kc; ++kk) {
                const float2 a = widen<TA, DT>(As[threadIdx.x * kc + kk]);
#pragma unroll
                for (int j = 0; j < NC; ++j) {
                    if (j < nc) {
                        const float2 bb = Bs[kk][j];
                        acc[j].x = fmaf(a.x, bb.x, fmaf(-a.y, bb.y, acc[j].x));
                        acc[j].y = fmaf(a.x, bb.y, fmaf(a.y, bb.x, acc[j].y));
                    }
                }
            }
        }
        if (((k0 + KC) % kFlushK) == 0 || k0 + KC >= K) {
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                tot[j].x += acc[j].x;
                tot[j].y += acc[j].y;
                acc[j] = make_float2(0.f, 0.f);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = make_float2((float)tot[j].x, (float)tot[j].y);
    // every thread stays to the end: the maximum is reduced over the warp and
    // recorded with one atomic per warp (one per thread serialises on a
    // single address for steps of 2^30 rows)
    const bool active = threadIdx.x < rows;
    const int64_t m = m0 + threadIdx.x;
    TC *crow = Cb + m * N + n0;
    if constexpr (std::is_same<TC, float2>::value) {
        // complex64 result: no rounding to complex-half, no scaling (e = 0);
        // in complex-half plans its exponent and maximum feed later steps
        float mx = 0.f;
#pragma unroll
        for (int j = 0; j < NC; ++j)
            if (active && j < nc) {
                crow[j] = acc[j];
                mx = fmaxf(mx, fmaxf(fabsf(acc[j].x), fabsf(acc[j].y)));
            }
        if (sr.tmax) {
            if (sr.texp && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
                sr.texp[sr.meta_c] = sr.texp[sr.meta_a] + sr.texp[sr.meta_b];
            mx = warp_max(mx);
            if (sr.out_max && (threadIdx.x & 31) == 0) atomic_max_nonneg(sr.out_max, mx);
        }
    } else {
        // power-of-two scaling (exact): e from the operands' recorded maxima
        int e;
        if (sr.scale_off) e = 0;
        else if (sr.tmax) e = min(120, scale_exponent(sr.tmax[sr.meta_a], sr.tmax[sr.meta_b], lk) + sr.headroom);
        else e = sr.fixed_exp;
        if (sr.texp && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
            sr.texp[sr.meta_c] = sr.texp[sr.meta_a] + sr.texp[sr.meta_b] + e;
        const float s = exp2i(e);
        float mx = 0.f;
#pragma unroll
        for (int j = 0; j < NC; ++j)
            if (active && j < nc) {
                const auto h = LpT<DT>::from_f2(make_float2(acc[j].x * s, acc[j].y * s));
                crow[j] = h;
                const float2 f = LpT<DT>::to_f2(h);
                mx = fmaxf(mx, fmaxf(fabsf(f.x), fabsf(f.y)));
            }
        mx = warp_max(mx);
        if ((threadIdx.x & 31) == 0) {
            if (sr.out_max) atomic_max_nonneg(sr.out_max, mx);
            if (DT == TN_F16 && sr.err && !(mx <= 65504.0f)) atomicOr(sr.err, 2);
        }
    }
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
#define TN_ROWS_CASE(NCV)                                                                        \
    {                                                                                             \
        dim3 g((unsigned)gx, (unsigned)((N + NCV - 1) / NCV), (unsigned)batch);                   \
        gemm_rows_kernel<TA, TB, TC, NCV, DT><<<g, kRows, 0, s>>>(                                \
            (const TA *)A, (const TB *)B, (TC *)C, lm, ln, lk, sa, sb, sc, sr, za, zb);           \
        break;                                                                                    \
    }
    switch (N >= 16 ? 16 : N) {
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
// 64x64 output tile per block of 256 threads, 4x4 complex outputs per
// thread, K in chunks of 16 staged through shared memory.  Needs M, N >= 64.
// LONGK: FP32 partial sums over kFlushK terms added into FP64 (for K >
// 2^12, where one FP32 running sum would lose ~sqrt(K) ulps); the short-K
// instance keeps the FP32 sum and half the registers.
template <int BM, int BN, int BK, bool LONGK>
__global__ void __launch_bounds__(256) gemm_tiled_c64_kernel(
    const float2 *__restrict__ A, const float2 *__restrict__ B, float2 *__restrict__ C, int lm,
    int ln, int lk, int64_t sa, int64_t sb, int64_t sc, const int32_t *za, const int32_t *zb) {
    constexpr int TM = BM / 16, TN = BN / 16;
    __shared__ float2 As[BK][BM + 1];
    __shared__ float2 Bs[BK][BN];
    const int N = 1 << ln, K = 1 << lk;
    const int64_t b = blockIdx.z;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const float2 *Ab = A + (za ? (int64_t)za[b] : b) * sa + m0 * K;
    const float2 *Bb = B + (zb ? (int64_t)zb[b] : b) * sb + n0;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float2 acc[TM][TN];
    double2 tot[LONGK ? TM : 1][LONGK ? TN : 1];   // FP64 sum of the FP32 partials
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            acc[i][j] = make_float2(0.f, 0.f);
            if constexpr (LONGK) tot[i][j] = make_double2(0.0, 0.0);
        }
    // the next K slice is loaded into registers while the current one is
    // multiplied out of shared memory
    constexpr int EA = BM * BK / 256, EB = BK * BN / 256;
    static_assert(EA * 256 == BM * BK && EB * 256 == BK * BN, "tile not a multiple of the block");
    float2 ra[EA], rb[EB];
    auto load_regs = [&](int k0) {
#pragma unroll
        for (int e = 0; e < EA; ++e) {
            const int i = threadIdx.x + 256 * e, r = i / BK, kk = i % BK;
            ra[e] = Ab[(int64_t)r * K + k0 + kk];
        }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
            const int i = threadIdx.x + 256 * e, kk = i / BN, c = i % BN;
            rb[e] = Bb[(int64_t)(k0 + kk) * N + c];
        }
    };
    load_regs(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int e = 0; e < EA; ++e) {
            const int i = threadIdx.x + 256 * e;
            As[i % BK][i / BK] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
            const int i = threadIdx.x + 256 * e;
            Bs[i / BN][i % BN] = rb[e];
        }
        __syncthreads();
        if (k0 + BK < K) load_regs(k0 + BK);
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            float2 a[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    acc[i][j].x = fmaf(a[i].x, bv[j].x, fmaf(-a[i].y, bv[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(a[i].x, bv[j].y, fmaf(a[i].y, bv[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
        if constexpr (LONGK) {
            if (((k0 + BK) % kFlushK) == 0 || k0 + BK >= K) {
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        tot[i][j].x += acc[i][j].x;
                        tot[i][j].y += acc[i][j].y;
                        acc[i][j] = make_float2(0.f, 0.f);
                    }
            }
        }
    }
    float2 *Cb = C + b * sc + m0 * N + n0;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            float2 v = acc[i][j];
            if constexpr (LONGK) v = make_float2((float)tot[i][j].x, (float)tot[i][j].y);
            Cb[(int64_t)(ty * TM + i) * N + tx + 16 * j] = v;
        }
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
    int e = 0;
    if (!OUT_C64) {
        if (sr.scale_off) e = 0;
        else if (sr.tmax) e = min(120, scale_exponent(sr.tmax[sr.meta_a], sr.tmax[sr.meta_b], lk) + sr.headroom);
        else e = sr.fixed_exp;
    }
    if (sr.texp && blockIdx.x == 0 && threadIdx.x == 0)
        sr.texp[sr.meta_c] = sr.texp[sr.meta_a] + sr.texp[sr.meta_b] + e;
    const float sc = exp2i(e);
    float mx = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int p = 0; p < split; ++p) {
            const float2 v = partial[(int64_t)p * n + i];
            re += v.x;
            im += v.y;
        }
        if constexpr (OUT_C64) {
            const float2 w = make_float2((float)re, (float)im);
            reinterpret_cast<float2 *>(C)[i] = w;
            mx = fmaxf(mx, fmaxf(fabsf(w.x), fabsf(w.y)));
        } else {
            const auto h = LpT<DT>::from_f2(make_float2((float)re * sc, (float)im * sc));
            reinterpret_cast<typename LpT<DT>::T2 *>(C)[i] = h;
            const float2 f = LpT<DT>::to_f2(h);
            mx = fmaxf(mx, fmaxf(fabsf(f.x), fabsf(f.y)));
        }
    }
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0 && sr.out_max) atomic_max_nonneg(sr.out_max, mx);
    if (!OUT_C64 && DT == TN_F16 && sr.err && (threadIdx.x & 31) == 0 && !(mx <= 65504.0f))
        atomicOr(sr.err, 2);
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
// amp[j] (+)= sum over batch index t in [t_lo, t_hi), ascending, of
// c * F[idx(j, t)] * 2^-E (FP64; one slice added at a time).  F is stored
// complex64 or complex-half; c is the product of the per-step rounding
// compensations of the complex-half plan (1 otherwise).
// Recomputation: the op's split outputs are absent from F; thread j covers
// the amplitude whose split bits are split_val and whose other bits, in
// order, are j's bits.
template <typename TF, int DT>
__global__ void slice_sum_kernel(const TF *__restrict__ F, const SumOp op, double2 *amps,
                                 int n_open, int t_lo, int t_hi, int overwrite,
                                 const int32_t *texp, const double2 *__restrict__ stepcorr,
                                 int n_steps, uint64_t split_mask, uint64_t split_val) {
    const int64_t n = (int64_t)1 << (n_open - op.n_split);
    const int64_t jf = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (jf >= n) return;
    int64_t base = 0, j = (int64_t)split_val;
    for (int t = 0, u = 0; t < n_open; ++t) {
        if ((split_mask >> t) & 1) continue;
        if ((jf >> u) & 1) {
            base |= (int64_t)1 << op.open_pos[t];
            j |= (int64_t)1 << t;
        }
        ++u;
    }
    const int E = texp ? texp[op.meta] : 0;
    double cr = 1.0, ci = 0.0;
    for (int k = 0; k < n_steps; ++k) {
        const double2 f = stepcorr[k];
        const double nr = cr * f.x - ci * f.y;
        ci = cr * f.y + ci * f.x;
        cr = nr;
    }
    double2 a = overwrite ? make_double2(0.0, 0.0) : amps[j];
    for (int t = t_lo; t < t_hi; ++t) {
        int64_t idx = base;
        for (int q = 0; q < op.n_batch; ++q)
            if ((t >> q) & 1) idx |= (int64_t)1 << op.batch_pos[q];
        const float2 v = widen<TF, DT>(F[idx]);
        double re = ldexp((double)v.x, -E), im = ldexp((double)v.y, -E);
        if (n_steps > 0) {
            const double nre = cr * re - ci * im;
            im = cr * im + ci * re;
            re = nre;
        }
        a.x += re;
        a.y += im;
    }
    amps[j] = a;
}

cudaError_t launch_slice_sum(const void *F, int dtype, const SumOp &op, double2 *amps, int n_open,
                             int t_lo, int t_hi, int overwrite, const int32_t *texp,
                             const double2 *stepcorr, int n_steps, uint64_t split_val, cudaStream_t s) {
    if (op.n_split < 0 || op.n_split > 8 || op.n_split > n_open) return cudaErrorInvalidValue;
    uint64_t split_mask = 0;
    for (int i = 0; i < op.n_split; ++i) split_mask |= 1ull << op.split_t[i];
    if ((split_val & ~split_mask) != 0) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)1 << (n_open - op.n_split);
    const int threads = 256;
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

}  // namespace tn
