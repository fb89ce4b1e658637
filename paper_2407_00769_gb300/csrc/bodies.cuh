// Device bodies of the SIMT kernels (leaf preparation, permutations, B'
// builds, CUDA-core GEMMs, split-K reduction, FP64 slice sum), written once
// and called from two places: the stand-alone kernels of kernels.cu (one
// launch per op, block coordinates from blockIdx) and the work-queue kernel
// of queue.cu (many ops in one persistent launch, block coordinates from the
// queue item).  Each body takes its block coordinates, its thread index and
// its shared memory explicitly, and synchronizes through the Sync policy it
// is instantiated with (__syncthreads in a stand-alone kernel, a named
// barrier over the participating threads in the queue), so both paths run
// the same arithmetic in the same order and produce the same bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "kernels.cuh"

namespace tn {

// --------------------------------------------------------- sync policies --
struct SyncBlock {
    __device__ __forceinline__ static void sync() { __syncthreads(); }
};
template <int ID, int NT>
struct SyncNamed {
    __device__ __forceinline__ static void sync() { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NT) : "memory"); }
};

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

// operand conversion: complex64 as is, complex-half widened to FP32
template <typename T, int DT>
__device__ __forceinline__ float2 widen(T v) {
    if constexpr (std::is_same<T, float2>::value) return v;
    else return LpT<DT>::to_f2(v);
}

// ------------------------------------------------------------- leaf prep --
// One warp per leaf.  Output element o (over the kept legs) reads input
// element in(o) = kept bits placed at keep_pos, fixed legs at the value of
// their slice-id bit (slice decoding: bit j of the slice id is sliced edge
// j's value).  Converts complex128 -> complex64 (RN); tmax (complex-half
// plans) records the leaf's largest component for the scaling of the steps
// that consume it.
__device__ __forceinline__ void leaf_warp_body(const LeafJob &j, const double2 *store, char *ws,
                                               int64_t slice_base, float *tmax, int32_t *texp, int lane) {
    const int n_out = 1 << j.rank_out;
    float m = 0.0f;
    for (int o = lane; o < n_out; o += 32) {
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
        if (lane == 0) {
            tmax[j.meta] = m;
            texp[j.meta] = 0;
        }
    }
}

// --------------------------------------------------------------- permute --
// Generic bit-permute tile (tile_bits <= 10): the block reads its tile in
// input order (coalesced), stages it in shared memory (tile: 1024 + 32
// elements), and writes it in output order (coalesced).  Tile `tid_tile`
// supplies the outer bits.  Pure data movement: bit-exact.
template <typename T, class Sync>
__device__ __forceinline__ void permute_tile_body(const T *in, T *out, const PermParams &p, int64_t tid_tile,
                                                  int tid, int nthr, T *tile) {
    int64_t bin = 0, bout = 0;
    for (int k = 0; k < p.n_outer; ++k)
        if ((tid_tile >> k) & 1) {
            bin |= (int64_t)1 << p.outer_in[k];
            bout |= (int64_t)1 << p.outer_out[k];
        }
    const int n = 1 << p.tile_bits;
    const int lo_mask_in = (1 << p.lin) - 1;
    for (int e = tid; e < n; e += nthr) {
        const int64_t off = bin + (e & lo_mask_in) + p.rd_hi_off[e >> p.lin];
        tile[e + (e >> 5)] = in[off];
    }
    Sync::sync();
    const int lo_mask_out = (1 << p.lout) - 1;
    for (int f = tid; f < n; f += nthr) {
        const int fl = f & lo_mask_out, fh = f >> p.lout;
        const int e = p.wr_lo_e[fl] | p.wr_hi_e[fh];
        out[bout + fl + p.wr_hi_off[fh]] = tile[e + (e >> 5)];
    }
}

// Fast path for tensors of rank >= 10 (256 threads): the tile is always
// 2^10 elements (32 contiguous input elements x 32 contiguous output
// elements), and the position of an element inside its tile is the same for
// every tile, so each thread works out once where its 4 elements come from
// and go to; per tile only the tile's base offsets change (from 8-bit lookup
// tables).  Each thread moves its 4 elements with one 16-byte (4-byte
// elements) or two (8-byte elements) vector loads and stores.  The body walks
// tiles first, first + step, ... below end, NT per iteration (NT 16-byte
// loads in flight per thread).
//
// EXPAND (complex-half only): instead of the permuted tensor, write the
// padded real operand of the tensor-core GEMM (Sec. 3.3, Eq. 6): the
// permuted order is [batch][N][K] complex and element (b, n, k) = (re, im)
// goes to B'[b][2n][k] = (re, -im) and B'[b][2n+1][k] = (im, re) (pairs of
// halves; np rows per batch).
struct ExpandArgs {
    int32_t lk, ln, np;
};

template <typename T, int NT = 2>
struct PermTiledSmem {
    T tile[NT][1024 + 32];
    int64_t s_bin[4][256], s_bout[4][256];
};

template <typename T, bool EXPAND, class Sync, int NT = 2>
__device__ __forceinline__ void permute_tiled_body(const T *in, void *out_, const PermParams &p, int64_t first,
                                                   int64_t end, int64_t step, ExpandArgs ex, int tid,
                                                   PermTiledSmem<T, NT> &sm) {
    for (int i = tid; i < 1024; i += 256) {
        const int level = i >> 8, v = i & 255;
        int64_t bi = 0, bo = 0;
        for (int b = 0; b < 8; ++b) {
            const int k = level * 8 + b;
            if (k < p.n_outer && ((v >> b) & 1)) {
                bi |= (int64_t)1 << p.outer_in[k];
                bo |= (int64_t)1 << p.outer_out[k];
            }
        }
        sm.s_bin[level][v] = bi;
        sm.s_bout[level][v] = bo;
    }
    // this thread's 4 elements: read-order e0..e0+3, write-order f0..f0+3
    const int e0 = tid * 4;
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
    Sync::sync();
    for (int64_t t0 = first; t0 < end; t0 += NT * step) {
        T v[NT][4];
#pragma unroll
        for (int h = 0; h < NT; ++h) {
            const int64_t t = t0 + h * step;
            if (t >= end) break;
            const int64_t bin = sm.s_bin[0][t & 255] + sm.s_bin[1][(t >> 8) & 255] +
                                sm.s_bin[2][(t >> 16) & 255] + sm.s_bin[3][(t >> 24) & 255];
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
        for (int h = 0; h < NT; ++h) {
            if (t0 + h * step >= end) break;
#pragma unroll
            for (int j = 0; j < 4; ++j) sm.tile[h][rd_slot[j]] = v[h][j];
        }
        Sync::sync();
#pragma unroll
        for (int h = 0; h < NT; ++h) {
            const int64_t t = t0 + h * step;
            if (t >= end) break;
            const int64_t bout = sm.s_bout[0][t & 255] + sm.s_bout[1][(t >> 8) & 255] +
                                 sm.s_bout[2][(t >> 16) & 255] + sm.s_bout[3][(t >> 24) & 255];
            T w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = sm.tile[h][wr_slot[j]];
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
        Sync::sync();
    }
}

// ------------------------------------------------------------------ bprep --
// B already in [batch][N][K] order (complex-half, K >= 4) -> B' as a
// stream: unit u covers 4 consecutive k of one row pair (b, pr) of B'
// (pr < N: B row (b, pr) gives B' rows 2 pr = (re, -im) and 2 pr + 1 =
// (im, re); pr >= N: the zero rows that pad B' to np rows).  One 16-byte
// load and two 16-byte stores per unit, U units in flight per thread.
// Units u = first, first + step, ... < end.
template <int U>
__device__ __forceinline__ void bprep_stream_body(const uint4 *B, uint4 *Bp, int lk, int ln, int np, int64_t first,
                                                  int64_t end, int64_t step) {
    const int lq = lk - 2;                      // log2 of 16-byte units per row
    const int half = np >> 1;                   // row pairs of B' per batch entry
    const int N = 1 << ln;
    for (int64_t u0 = first; u0 < end; u0 += (int64_t)U * step) {
        uint4 x[U];
        int64_t dst[U];
        bool live[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int64_t u = u0 + (int64_t)j * step;
            x[j] = make_uint4(0u, 0u, 0u, 0u);
            dst[j] = -1;
            live[j] = false;
            if (u < end) {
                const int64_t q = u & (((int64_t)1 << lq) - 1);
                const int64_t row = u >> lq;           // b * half + pr
                const int pr = (int)(row % half);
                const int64_t b = row / half;
                live[j] = pr < N;
                if (live[j]) x[j] = B[(((b << ln) + pr) << lq) + q];
                dst[j] = ((b * np + 2 * pr) << lq) + q;
            }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (dst[j] < 0) continue;
            const uint4 w = x[j];
            uint4 r0 = make_uint4(0u, 0u, 0u, 0u), r1 = r0;
            if (live[j]) {
                // (re, -im): flip the sign bit of the high half; (im, re): swap halves
                r0 = make_uint4(w.x ^ 0x80000000u, w.y ^ 0x80000000u, w.z ^ 0x80000000u, w.w ^ 0x80000000u);
                r1 = make_uint4(__byte_perm(w.x, 0, 0x1032), __byte_perm(w.y, 0, 0x1032),
                                __byte_perm(w.z, 0, 0x1032), __byte_perm(w.w, 0, 0x1032));
            }
            Bp[dst[j]] = r0;
            Bp[dst[j] + ((int64_t)1 << lq)] = r1;
        }
    }
}

// B (complex-half, any mode order) -> B' by a direct gather: target complex
// index bits [batch][N][K] (LSB = k bit 0); for target bit t the input bit
// position is p.outer_in[t].  Elements i = first, first + step, ... < end of
// the uint32 pairs of B'.
__device__ __forceinline__ void bprep_gather_body(const uint32_t *B, uint32_t *Bp, int lk, int ln, int np,
                                                  const PermParams &p, int rank, int64_t first, int64_t end,
                                                  int64_t step) {
    const int K = 1 << lk, N = 1 << ln;
    for (int64_t i = first; i < end; i += step) {
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

// Complex64 B (a small tensor) -> B' in complex-half, one block of NT
// threads: every element is rounded to the plan's dtype here, and the
// rounding's component along B, alpha = <B, B~ - B> / <B, B>, is measured
// (FP64, fixed order) so the final sum can divide the factor (1 + alpha) out
// exactly (the network is linear in B): corr = 1 / (1 + alpha).  The FP64
// sums follow one fixed order whatever NT is: VT virtual threads (v takes
// elements v, v + VT, ...), then a tree over the VT partial sums; each real
// thread plays VT / NT of them.
template <int VT>
struct BprepC64Smem {
    double sh[3][VT];
    float smax[VT];
};

// Exact power-of-two scale 2^bshift bringing max |B| = mb to [2^11, 2^12].
__device__ __forceinline__ int bprep_c64_shift(float mb, int scale_off) {
    int bshift = 0;
    if (!scale_off && mb > 0.0f && isfinite(mb)) {
        int x;
        const float f = frexpf(mb, &x);
        bshift = 12 - ((f == 0.5f) ? x - 1 : x);
        bshift = max(-120, min(120, bshift));
    }
    return bshift;
}

// Virtual thread v of VT: the elements v, v + VT, ... of B' (written), with
// their FP64 sums (fixed order) and the maximum of the rounded values.
template <int DT, int VT>
__device__ __forceinline__ void bprep_c64_vthread(const float2 *B, uint32_t *Bp, int lk, int ln, int np, int64_t total,
                                                  const PermParams &p, int rank, float scale, int v, double &nr,
                                                  double &ni, double &den, float &bmax) {
    using L = LpT<DT>;
    const int K = 1 << lk, N = 1 << ln;
    bmax = 0.0f;
    nr = 0.0, ni = 0.0, den = 0.0;
    for (int64_t i = v; i < total; i += VT) {
        const int k = (int)(i % K);
        const int64_t row = i / K;
        const int rr = (int)(row % np);
        const int64_t b = row / np;
        const int n = rr >> 1, co = rr & 1;
        uint32_t val = 0;
        if (n < N) {
            const int64_t tidx = ((b * N + n) << lk) | k;
            int64_t src = 0;
            for (int t = 0; t < rank; ++t)
                if ((tidx >> t) & 1) src |= (int64_t)1 << p.outer_in[t];
            const float2 x0 = B[src];
            const float2 x = make_float2(x0.x * scale, x0.y * scale);
            const typename L::T2 h = L::from_f2(x);
            const uint32_t u = *reinterpret_cast<const uint32_t *>(&h);
            val = co == 0 ? (u ^ 0x80000000u) : __byte_perm(u, 0, 0x1032);
            if (co == 0) {
                const float2 r = L::to_f2(h);
                bmax = fmaxf(bmax, fmaxf(fabsf(r.x), fabsf(r.y)));
                const double dr = (double)r.x - x.x, di = (double)r.y - x.y;
                nr += (double)x.x * dr + (double)x.y * di;     // Re conj(x) d
                ni += (double)x.x * di - (double)x.y * dr;     // Im conj(x) d
                den += (double)x.x * x.x + (double)x.y * x.y;
            }
        }
        Bp[i] = val;
    }
}

// The tree over the VT partials in sm (pairs x, x + w for w = VT/2 .. 1) and
// the results: tmax / texp of B', and corr = 1 / (1 + alpha).
template <int NT, int VT, class Sync>
__device__ __forceinline__ void bprep_c64_finish(double2 *corr, float *tmax, int32_t *texp, int meta_src,
                                                 int meta_dst, int bshift, int tid, BprepC64Smem<VT> &sm) {
    Sync::sync();
    for (int w = VT / 2; w > 0; w >>= 1) {
        for (int x = tid; x < w; x += NT) {
            for (int q = 0; q < 3; ++q) sm.sh[q][x] += sm.sh[q][x + w];
            sm.smax[x] = fmaxf(sm.smax[x], sm.smax[x + w]);
        }
        Sync::sync();
    }
    if (tid == 0) {
        tmax[meta_dst] = sm.smax[0];
        texp[meta_dst] = texp[meta_src] + bshift;
    }
    if (tid == 0 && corr) {
        double fr = 1.0, fi = 0.0;
        if (sm.sh[2][0] > 0.0) {
            // 1 / (1 + alpha)
            const double ar = 1.0 + sm.sh[0][0] / sm.sh[2][0], ai = sm.sh[1][0] / sm.sh[2][0];
            const double d = ar * ar + ai * ai;
            fr = ar / d;
            fi = -ai / d;
        }
        *corr = make_double2(fr, fi);
    }
}

template <int DT, int NT, int VT, class Sync>
__device__ __forceinline__ void bprep_c64_body(const float2 *B, uint32_t *Bp, int lk, int ln, int lb, int np,
                                               const PermParams &p, int rank, double2 *corr, float *tmax,
                                               int32_t *texp, int meta_src, int meta_dst, int scale_off, int tid,
                                               BprepC64Smem<VT> &sm) {
    static_assert(VT % NT == 0, "virtual threads must be a multiple of the block");
    const int64_t total = ((int64_t)np << lk) << lb;
    const int bshift = bprep_c64_shift(tmax[meta_src], scale_off);
    const float scale = __int_as_float((127 + bshift) << 23);
    for (int v = tid; v < VT; v += NT) {
        double nr, ni, den;
        float bmax;
        bprep_c64_vthread<DT, VT>(B, Bp, lk, ln, np, total, p, rank, scale, v, nr, ni, den, bmax);
        sm.sh[0][v] = nr;
        sm.sh[1][v] = ni;
        sm.sh[2][v] = den;
        sm.smax[v] = bmax;
    }
    bprep_c64_finish<NT, VT, Sync>(corr, tmax, texp, meta_src, meta_dst, bshift, tid, sm);
}

// ----------------------------------------------------------- rows GEMMs --
// C[b][m][n] = sum_k A[b][m][k] B[b][k][n].  A block of kRows threads owns
// kRows consecutive rows (one per thread) and NC consecutive columns (block
// coordinate by); the A tile is staged through shared memory with coalesced
// 16-byte loads (its rows are contiguous), B's column chunk sits in shared
// memory as FP32 complex.  K is walked in chunks of KC.
constexpr int kRows = 128;
constexpr int kKC = 32;
constexpr int kFlushK = 256;   // FP32 terms per partial sum before the FP64 add

template <typename TA, int NC>
struct RowsSmem {
    // A tile rows padded to kc + 1 elements: each thread reads its own row,
    // so an unpadded power-of-two row stride would put all 32 lanes of a
    // warp on one bank
    TA As[kRows * (kKC + 1)];
    float2 Bs[kKC][NC];
};

// Operand and result storage may differ (complex-half plans keep small
// tensors in complex64): TA, TB, TC are float2 or the plan's complex-half
// type, DT the plan's dtype.
template <typename TA, typename TB, typename TC, int NC, int DT, class Sync>
__device__ __forceinline__ void rows_body(const TA *A, const TB *B, TC *C, int lm, int ln, int lk, int64_t sa,
                                          int64_t sb, int64_t sc, const ScaleRef &sr, const int32_t *za,
                                          const int32_t *zb, int64_t bx, int by, int64_t bz, int tid,
                                          RowsSmem<TA, NC> &sm, float &mx_run) {
    constexpr int KC = kKC;
    TA *As = sm.As;
    const int64_t M = (int64_t)1 << lm;
    const int N = 1 << ln, K = 1 << lk;
    const int64_t b = bz;
    const int64_t m0 = bx * kRows;
    const int n0 = by * NC;
    const int nc = min(NC, N);
    // sparse-state gathers: operand chunks by index instead of by batch entry
    const TA *Ab = A + (za ? (int64_t)za[b] : b) * sa;
    const TB *Bb = B + (zb ? (int64_t)zb[b] : b) * sb;
    TC *Cb = C + b * sc;
    const int rows = (int)min((int64_t)kRows, M - m0);
    // FP32 partial sums over at most kFlushK terms, added into FP64: a long
    // FP32 running sum would lose ~sqrt(K) ulps (2^23-term steps occur).
    // With K <= kFlushK the one partial is the sum (the FP64 round trip is
    // exact), and the FP64 pipe -- a small fraction of the FP32 rate on this
    // part -- is left out: it bounded steps of 2^22 rows and K = 4
    const bool longk = K > kFlushK;
    float2 acc[NC];
    double2 tot[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        acc[j] = make_float2(0.f, 0.f);
        tot[j] = make_double2(0.0, 0.0);
    }
    // K and KC are powers of two: every chunk holds kc = min(KC, K) terms
    const int lkc = min(lk, 5);
    static_assert(KC == 32, "lkc assumes 32-term chunks");
    const int ld = (1 << lkc) + 1;
    for (int k0 = 0; k0 < K; k0 += KC) {
        const int kc = 1 << lkc;
        Sync::sync();
        // A tile: rows x kc elements, row r at As[r * ld]; when kc == K the
        // tile is contiguous in memory and read with 16-byte loads
        {
            constexpr int per16 = 16 / (int)sizeof(TA);
            const int total = rows * kc;
            if (kc == K && (total % per16) == 0) {
                const uint4 *src = reinterpret_cast<const uint4 *>(Ab + m0 * K);
                for (int i = tid; i < total / per16; i += kRows) {
                    const uint4 x = src[i];
                    const TA *xv = reinterpret_cast<const TA *>(&x);
#pragma unroll
                    for (int u = 0; u < per16; ++u) {
                        const int e = i * per16 + u;
                        As[(e >> lkc) * ld + (e & (kc - 1))] = xv[u];
                    }
                }
            } else {
                for (int i = tid; i < total; i += kRows) {
                    const int r = i >> lkc, kk = i & (kc - 1);
                    As[r * ld + kk] = Ab[(m0 + r) * K + k0 + kk];
                }
            }
        }
        for (int i = tid; i < kc * nc; i += kRows) {
            const int kk = i / nc, j = i % nc;
            sm.Bs[kk][j] = widen<TB, DT>(Bb[(int64_t)(k0 + kk) * N + n0 + j]);
        }
        Sync::sync();
        if (tid < rows) {
            for (int kk = 0; kk < kc; ++kk) {
                const float2 a = widen<TA, DT>(As[tid * ld + kk]);
#pragma unroll
                for (int j = 0; j < NC; ++j) {
                    if (j < nc) {
                        const float2 bb = sm.Bs[kk][j];
                        acc[j].x = fmaf(a.x, bb.x, fmaf(-a.y, bb.y, acc[j].x));
                        acc[j].y = fmaf(a.x, bb.y, fmaf(a.y, bb.x, acc[j].y));
                    }
                }
            }
        }
        if (longk && (((k0 + KC) % kFlushK) == 0 || k0 + KC >= K)) {
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                tot[j].x += acc[j].x;
                tot[j].y += acc[j].y;
                acc[j] = make_float2(0.f, 0.f);
            }
        }
    }
    if (longk) {
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = make_float2((float)tot[j].x, (float)tot[j].y);
    } else {
        // + 0: a -0 partial becomes +0, as 0.0 + (-0.0) does in the FP64 sum
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = make_float2(acc[j].x + 0.0f, acc[j].y + 0.0f);
    }
    // the maximum of the stored values goes to mx_run (this thread's running
    // maximum); rows_flush records it once per warp after all of a CTA's row
    // blocks (an atomic per thread, or per warp and row block, serialises on
    // one address for steps of 2^22+ rows)
    const bool active = tid < rows;
    const bool first_block = bx == 0 && by == 0 && bz == 0 && tid == 0;
    const int64_t m = m0 + tid;
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
            if (sr.texp && first_block) sr.texp[sr.meta_c] = sr.texp[sr.meta_a] + sr.texp[sr.meta_b];
            mx_run = fmaxf(mx_run, mx);
        }
    } else {
        // power-of-two scaling (exact): e from the operands' recorded maxima
        int e;
        if (sr.scale_off) e = 0;
        else if (sr.tmax) e = min(120, scale_exponent(sr.tmax[sr.meta_a], sr.tmax[sr.meta_b], lk) + sr.headroom);
        else e = sr.fixed_exp;
        if (sr.texp && first_block) sr.texp[sr.meta_c] = sr.texp[sr.meta_a] + sr.texp[sr.meta_b] + e;
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
        mx_run = fmaxf(mx_run, mx);
    }
}

// Record a rows GEMM thread's running maximum (rows_body's mx_run): reduced
// over the warp, one atomic per warp (the maximum is exact and order-free);
// for complex-half results also the FP16 overflow flag.  Every thread of the
// warp calls it.
template <typename TC, int DT>
__device__ __forceinline__ void rows_flush(const ScaleRef &sr, float mx, int tid) {
    if constexpr (std::is_same<TC, float2>::value) {
        if (!sr.tmax) return;
        mx = warp_max(mx);
        if (sr.out_max && (tid & 31) == 0) atomic_max_nonneg(sr.out_max, mx);
    } else {
        mx = warp_max(mx);
        if ((tid & 31) == 0) {
            if (sr.out_max) atomic_max_nonneg(sr.out_max, mx);
            if (DT == TN_F16 && sr.err && !(mx <= 65504.0f)) atomicOr(sr.err, 2);
        }
    }
}

// ---------------------------------------------------------- tiled c64 --
// BM x BN output tile per block of 256 threads, 4x4 complex outputs per
// thread, K in chunks of BK staged through shared memory.  Needs M, N >= 64.
// LONGK: FP32 partial sums over kFlushK terms added into FP64 (for K >
// 2^12, where one FP32 running sum would lose ~sqrt(K) ulps); the short-K
// instance keeps the FP32 sum and half the registers.
template <int BM, int BN, int BK>
struct TiledC64Smem {
    float2 As[BK][BM + 1];
    float2 Bs[BK][BN];
};

template <int BM, int BN, int BK, bool LONGK, class Sync>
__device__ __forceinline__ void tiled_c64_body(const float2 *A, const float2 *B, float2 *C, int lm, int ln,
                                               int lk, int64_t sa, int64_t sb, int64_t sc, const int32_t *za,
                                               const int32_t *zb, int64_t bx, int by, int64_t bz, int tid,
                                               TiledC64Smem<BM, BN, BK> &sm) {
    (void)lm;
    constexpr int TM = BM / 16, TN = BN / 16;
    const int N = 1 << ln, K = 1 << lk;
    const int64_t b = bz;
    const int64_t m0 = bx * BM;
    const int n0 = by * BN;
    const float2 *Ab = A + (za ? (int64_t)za[b] : b) * sa + m0 * K;
    const float2 *Bb = B + (zb ? (int64_t)zb[b] : b) * sb + n0;
    const int tx = tid % 16, ty = tid / 16;
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
            const int i = tid + 256 * e, r = i / BK, kk = i % BK;
            ra[e] = Ab[(int64_t)r * K + k0 + kk];
        }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
            const int i = tid + 256 * e, kk = i / BN, c = i % BN;
            rb[e] = Bb[(int64_t)(k0 + kk) * N + c];
        }
    };
    load_regs(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int e = 0; e < EA; ++e) {
            const int i = tid + 256 * e;
            sm.As[i % BK][i / BK] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
            const int i = tid + 256 * e;
            sm.Bs[i / BN][i % BN] = rb[e];
        }
        Sync::sync();
        if (k0 + BK < K) load_regs(k0 + BK);
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            float2 a[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = sm.As[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = sm.Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    acc[i][j].x = fmaf(a[i].x, bv[j].x, fmaf(-a[i].y, bv[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(a[i].x, bv[j].y, fmaf(a[i].y, bv[j].x, acc[i][j].y));
                }
        }
        Sync::sync();
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

// --------------------------------------------------------- split-K reduce --
// Elements i = first, first + step, ... < end (<= n): the sum of the K parts' FP32
// partials in FP64 (part order), then the single-part epilogue's scaling and
// rounding.  first_block: writes the output exponent (once per op).
template <int DT, bool OUT_C64>
__device__ __forceinline__ void splitk_body(const float2 *partial, int split, void *C, int64_t n, int lk,
                                            const ScaleRef &sr, int64_t first, int64_t end, int64_t step,
                                            bool first_block, int tid) {
    int e = 0;
    if (!OUT_C64) {
        if (sr.scale_off) e = 0;
        else if (sr.tmax) e = min(120, scale_exponent(sr.tmax[sr.meta_a], sr.tmax[sr.meta_b], lk) + sr.headroom);
        else e = sr.fixed_exp;
    }
    if (sr.texp && first_block && tid == 0) sr.texp[sr.meta_c] = sr.texp[sr.meta_a] + sr.texp[sr.meta_b] + e;
    const float sc = exp2i(e);
    float mx = 0.f;
    for (int64_t i = first; i < end; i += step) {
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
    if ((tid & 31) == 0 && sr.out_max) atomic_max_nonneg(sr.out_max, mx);
    if (!OUT_C64 && DT == TN_F16 && sr.err && (tid & 31) == 0 && !(mx <= 65504.0f)) atomicOr(sr.err, 2);
}

// ------------------------------------------------------------- slice sum --
// amp[j] (+)= sum over batch index t in [t_lo, t_hi), ascending, of
// c * F[idx(j, t)] * 2^-E (FP64; one slice added at a time).  F is stored
// complex64 or complex-half; c is the product of the per-step rounding
// compensations of the complex-half plan (1 otherwise).
// Recomputation: the op's split outputs are absent from F; thread jf covers
// the amplitude whose split bits are split_val and whose other bits, in
// order, are jf's bits.
__device__ __forceinline__ double2 slice_corr(const double2 *stepcorr, int n_steps) {
    double cr = 1.0, ci = 0.0;
    for (int k = 0; k < n_steps; ++k) {
        const double2 f = stepcorr[k];
        const double nr = cr * f.x - ci * f.y;
        ci = cr * f.y + ci * f.x;
        cr = nr;
    }
    return make_double2(cr, ci);
}

// corr: slice_corr(stepcorr, n_steps), the same for every amplitude (one
// thread of a block computes it: FP64 runs at a small fraction of the FP32
// rate here)
template <typename TF, int DT>
__device__ __forceinline__ void slice_sum_body(const TF *F, const SumOp &op, double2 *amps, int n_open, int t_lo,
                                               int t_hi, int overwrite, const int32_t *texp, double2 corr,
                                               int n_steps, uint64_t split_mask, uint64_t split_val, int64_t jf) {
    const int64_t n = (int64_t)1 << (n_open - op.n_split);
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
    const double cr = corr.x, ci = corr.y;
    double2 a = overwrite ? make_double2(0.0, 0.0) : amps[j];
    // x 2^-E as one multiplication where 2^-E is a normal or subnormal double
    // (exact, the same value as ldexp); ldexp itself outside that range
    const bool mul = E >= -1000 && E <= 1000;
    const double sc = mul ? ldexp(1.0, -E) : 1.0;
    // the slices in order t_lo, t_lo + 1, ... (a fixed summation order); the
    // loads of 8 slices are issued before their adds so that their latencies
    // overlap instead of adding up
    constexpr int U = 8;
    for (int t0 = t_lo; t0 < t_hi; t0 += U) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u;
            if (t >= t_hi) break;
            int64_t idx = base;
            for (int q = 0; q < op.n_batch; ++q)
                if ((t >> q) & 1) idx |= (int64_t)1 << op.batch_pos[q];
            v[u] = widen<TF, DT>(F[idx]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (t0 + u >= t_hi) break;
            double re = mul ? (double)v[u].x * sc : ldexp((double)v[u].x, -E);
            double im = mul ? (double)v[u].y * sc : ldexp((double)v[u].y, -E);
            if (n_steps > 0) {
                const double nre = cr * re - ci * im;
                im = cr * im + ci * re;
                re = nre;
            }
            a.x += re;
            a.y += im;
        }
    }
    amps[j] = a;
}

}  // namespace tn
