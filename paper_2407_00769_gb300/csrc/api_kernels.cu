// Single-kernel entry points of the C ABI -- tn_permute, tn_gemm,
// tn_gemm_gather -- and the failure-detection self-tests: one contraction
// kernel (plus its B' build) per call, as the parity tests and the kernel
// benchmarks use them; the plan entry points are in api.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "plan.h"

using namespace tn;

namespace {

int fail(int code, const std::string &msg) { return record_error(code, msg); }

int cuda_fail(cudaError_t e, const char *where) {
    return fail(TN_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define TN_CUDA(call, where)                         \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

}  // namespace

extern "C" {

int tn_permute(const void *in, void *out, int32_t rank, const int32_t *perm, int32_t elem_bytes,
               void *stream) {
    if (!in || !out || !perm) return fail(TN_EINVAL, "NULL argument");
    if (rank < 0 || rank > 34) return fail(TN_EINVAL, "rank must be in 0..34");
    if (elem_bytes != 4 && elem_bytes != 8) return fail(TN_EINVAL, "elem_bytes must be 4 or 8");
    bool seen[kMaxRank] = {false};
    for (int i = 0; i < rank; ++i) {
        if (perm[i] < 0 || perm[i] >= rank || seen[perm[i]]) return fail(TN_EINVAL, "perm is not a permutation");
        seen[perm[i]] = true;
    }
    const PermParams pp = make_perm_params(rank, perm);
    cudaError_t e = launch_permute(in, out, pp, elem_bytes, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "tn_permute");
    return TN_OK;
}

int tn_gemm(int32_t dtype, const void *A, const void *B, void *C, int64_t M, int64_t N, int64_t K,
            int64_t batch, int32_t batch_a, int32_t batch_b, int32_t scale_exp, int32_t kernel,
            float *out_max, void *stream) {
    if (!A || !B || !C) return fail(TN_EINVAL, "NULL operand");
    auto lg = [](int64_t v) {
        int l = 0;
        while (l < 62 && ((int64_t)1 << l) < v) ++l;
        return (((int64_t)1 << l) == v) ? l : -1;
    };
    const int lm = lg(M), ln = lg(N), lk = lg(K);
    if (lm < 0 || ln < 0 || lk < 0 || lm > 34 || ln > 24 || lk > 24)
        return fail(TN_EINVAL, "M, N, K must be powers of two (M <= 2^34, N, K <= 2^24)");
    if (batch < 1 || batch > 65535) return fail(TN_EINVAL, "batch must be in 1..65535");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t sa = batch_a ? M * K : 0, sb = batch_b ? K * N : 0, sc = M * N;
    cudaError_t e;
    if (dtype == TN_C64) {
        int kk = kernel;
        if (kk < 0) kk = (lm >= 6 && ln >= 6 && lk >= 4) ? GK_C64_TILED : GK_C64_ROWS;
        if (kk == 9) {
            // tensor cores, TF32 in three parts (hi x hi + hi x lo + lo x hi)
            if (!tc_gemm_supported(lk, ln)) return fail(TN_EUNSUPPORTED, "tensor-core path needs K >= 8");
            const int np = std::max(16, (int)(2 * N));
            const int64_t abatch = batch_a ? batch : 1, bbatch = batch_b ? batch : 1;
            const size_t abytes = (size_t)abatch * M * K * 8, bbytes = (size_t)bbatch * np * K * 8;
            void *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
            TN_CUDA(cudaMallocAsync(&ah, abytes, s), "cudaMallocAsync");
            TN_CUDA(cudaMallocAsync(&al, abytes, s), "cudaMallocAsync");
            TN_CUDA(cudaMallocAsync(&bh, bbytes, s), "cudaMallocAsync");
            TN_CUDA(cudaMallocAsync(&bl, bbytes, s), "cudaMallocAsync");
            e = launch_split_tf32(A, ah, al, abatch * M * K * 2, s);
            if (e == cudaSuccess) e = launch_bprep_x3(B, bh, bl, lk, ln, bbatch, np, s);
            float *part = nullptr;
            if (e == cudaSuccess) {
                TcGemmDesc d;
                d.dtype = TN_C64;
                d.A = ah; d.A2 = al; d.Bp = bh; d.Bp2 = bl; d.C = C;
                d.lm = lm; d.ln = ln; d.lk = lk;
                d.batch = batch;
                d.batch_a = batch_a ? 1 : 0;
                d.batch_b = batch_b ? 1 : 0;
                d.np = np;
                d.x3 = 1;
                d.out_c64 = 1;
                const size_t pb = tc_split_bytes(lm, ln, lk, batch);
                if (pb) e = cudaMallocAsync((void **)&part, pb, s);
                d.partial = part;
                ScaleRef sr0{};
                sr0.out_max = out_max;
                if (e == cudaSuccess) e = launch_gemm_tc(d, sr0, nullptr, s);
            }
            if (part) cudaFreeAsync(part, s);
            cudaFreeAsync(ah, s);
            cudaFreeAsync(al, s);
            cudaFreeAsync(bh, s);
            cudaFreeAsync(bl, s);
        } else if (kk == GK_C64_TILED)
            e = launch_gemm_tiled_c64((const float2 *)A, (const float2 *)B, (float2 *)C, lm, ln, lk,
                                      batch, sa, sb, sc, 0, s);
        else if (kk == GK_C64_ROWS)
            e = launch_gemm_rows_c64((const float2 *)A, (const float2 *)B, (float2 *)C, lm, ln, lk,
                                     batch, sa, sb, sc, s);
        else
            return fail(TN_EINVAL, "kernel variant not valid for TN_C64");
    } else if (dtype == TN_FP8) {
        // E4M3 A [batch][M][K] and B [batch][K][N] complex, FP16 result
        if (kernel >= 0 && kernel != GK_LP_TC) return fail(TN_EINVAL, "TN_FP8 runs on the tensor cores only");
        if (!tc_gemm_supported_fp8(lk, ln)) return fail(TN_EUNSUPPORTED, "FP8 tensor-core path needs K >= 64");
        ScaleRef sr{};
        sr.fixed_exp = scale_exp;
        sr.out_max = out_max;
        const int np = std::max(16, (int)(2 * N));
        const int64_t bbatch = batch_b ? batch : 1;
        void *bp = nullptr;
        TN_CUDA(cudaMallocAsync(&bp, (size_t)np * 2 * K * bbatch, s), "cudaMallocAsync");
        e = launch_bprep_e4m3(B, bp, lk, ln, bbatch, np, s);
        if (e == cudaSuccess) {
            TcGemmDesc d;
            d.dtype = TN_F16;
            d.A = A; d.Bp = bp; d.C = C;
            d.lm = lm; d.ln = ln; d.lk = lk;
            d.batch = batch;
            d.batch_a = batch_a ? 1 : 0;
            d.batch_b = batch_b ? 1 : 0;
            d.np = np;
            d.fp8 = 1;
            const size_t pb = tc_split_bytes(lm, ln, lk, batch);
            if (pb) e = cudaMallocAsync((void **)&d.partial, pb, s);
            if (e == cudaSuccess) e = launch_gemm_tc(d, sr, nullptr, s);
            if (d.partial) cudaFreeAsync(d.partial, s);
        }
        cudaFreeAsync(bp, s);
    } else if (dtype == TN_F16 || dtype == TN_BF16) {
        ScaleRef sr{};
        sr.fixed_exp = scale_exp;
        sr.out_max = out_max;
        int kk = kernel;
        const bool pair = kk == 4;            // tensor cores on CTA pairs
        const bool half_k = kk == 5;          // tensor cores, 64-byte K chunks
        const bool bres = kk == 6 || kk == 7; // tensor cores, B' slice resident in shared memory
        const bool tma_store = kk == 7;       // ... and C tiles written by TMA stores
        const bool staged = kk == 8;          // tensor cores, C through per-warp staging
        if (pair || half_k || bres || staged) kk = GK_LP_TC;
        if (kk < 0) kk = tc_gemm_supported(lk, ln) ? GK_LP_TC : GK_LP_ROWS;
        if (kk == GK_LP_ROWS) {
            e = launch_gemm_rows_lp(dtype, A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s);
        } else if (kk == GK_LP_TC) {
            if (!tc_gemm_supported(lk, ln)) return fail(TN_EUNSUPPORTED, "tensor-core path needs K >= 8");
            const int np = std::max(16, (int)(2 * N));
            const int64_t bbatch = batch_b ? batch : 1;
            void *bp = nullptr;
            TN_CUDA(cudaMallocAsync(&bp, (size_t)np * 2 * K * 2 * bbatch, s), "cudaMallocAsync");
            e = launch_bprep(dtype, B, bp, lk, ln, bbatch, np, s);
            if (e == cudaSuccess) {
                TcGemmDesc d;
                d.dtype = dtype;
                d.A = A; d.Bp = bp; d.C = C;
                d.lm = lm; d.ln = ln; d.lk = lk;
                d.batch = batch;
                d.batch_a = batch_a ? 1 : 0;
                d.batch_b = batch_b ? 1 : 0;
                d.np = np;
                d.pair = pair ? 1 : 0;
                d.half_k = half_k ? 1 : 0;
                d.bres = bres ? 1 : 0;
                d.tma_store = tma_store ? 1 : 0;
                d.staged = staged ? 1 : 0;
                const size_t pb = tc_split_bytes(lm, ln, lk, batch);
                if (pb) e = cudaMallocAsync((void **)&d.partial, pb, s);
                if (e == cudaSuccess) e = launch_gemm_tc(d, sr, nullptr, s);
                if (d.partial) cudaFreeAsync(d.partial, s);
            }
            cudaFreeAsync(bp, s);
        } else {
            return fail(TN_EINVAL, "kernel variant not valid for complex-half");
        }
    } else {
        return fail(TN_EINVAL, "bad dtype");
    }
    if (e != cudaSuccess) return cuda_fail(e, "tn_gemm");
    return TN_OK;
}

int tn_gemm_gather(int32_t dtype, const void *A, int64_t m_a, const void *B, int64_t m_b, void *C,
                   int64_t m_n, int64_t M, int64_t N, int64_t K, const int32_t *index_a,
                   const int32_t *index_b, int32_t scheme, int32_t scale_exp, float *out_max,
                   int32_t *out_m_r, void *stream) {
    if (!A || !B || !C || !index_a || !index_b) return fail(TN_EINVAL, "NULL argument");
    if (dtype != TN_F16 && dtype != TN_BF16) return fail(TN_EINVAL, "tn_gemm_gather: dtype must be TN_F16 or TN_BF16");
    if (scheme != TN_GATHER_DIRECT && scheme != TN_GATHER_PADDED) return fail(TN_EINVAL, "bad scheme");
    auto lg = [](int64_t v) {
        int l = 0;
        while (l < 62 && ((int64_t)1 << l) < v) ++l;
        return (((int64_t)1 << l) == v) ? l : -1;
    };
    const int lm = lg(M), ln = lg(N), lk = lg(K);
    if (lm < 0 || ln < 0 || lk < 0 || lm > 30 || ln > 24) return fail(TN_EINVAL, "M, N, K must be powers of two");
    if (lk < 3 || lk > kSplitLog2K) return fail(TN_EUNSUPPORTED, "tn_gemm_gather needs 8 <= K <= 2^15");
    if (m_a < 1 || m_b < 1 || m_n < 1 || m_a > (1 << 30) || m_b > 65535 || m_n > (1 << 30))
        return fail(TN_EINVAL, "chunk counts: m_a, m_n in 1..2^30, m_b in 1..65535");
    for (int64_t n = 0; n < m_n; ++n) {
        if (index_a[n] < 0 || index_a[n] >= m_a || index_b[n] < 0 || index_b[n] >= m_b)
            return fail(TN_EINVAL, "index out of range at n = " + std::to_string(n));
        if (scheme == TN_GATHER_PADDED && n > 0 && index_a[n] < index_a[n - 1])
            return fail(TN_EINVAL, "TN_GATHER_PADDED needs a non-decreasing index_a");
    }
    // per tile-batch entry: A chunk, B' chunk, output chunk
    std::vector<int32_t> z;
    int64_t T = 0;
    int32_t m_r = 0;
    if (scheme == TN_GATHER_DIRECT) {
        T = m_n;
        z.resize(3 * T);
        for (int64_t n = 0; n < m_n; ++n) {
            z[n] = index_a[n];
            z[T + n] = index_b[n];
            z[2 * T + n] = (int32_t)n;
        }
    } else {
        std::vector<int32_t> count(m_a, 0);
        for (int64_t n = 0; n < m_n; ++n) m_r = std::max(m_r, ++count[index_a[n]]);
        T = m_a * (int64_t)m_r;
        if (T > (1LL << 31) - 1) return fail(TN_EINVAL, "padded index too large");
        z.assign(3 * T, 0);
        std::vector<int32_t> fill(m_a, 0);
        for (int64_t i = 0; i < m_a; ++i)
            for (int r = 0; r < m_r; ++r) {
                z[i * m_r + r] = (int32_t)i;
                z[2 * T + i * m_r + r] = -1;          // padded place: not stored
            }
        for (int64_t n = 0; n < m_n; ++n) {
            const int64_t i = index_a[n];
            const int64_t t = i * m_r + fill[i]++;
            z[T + t] = index_b[n];
            z[2 * T + t] = (int32_t)n;
        }
    }
    if (out_m_r) *out_m_r = m_r;
    cudaStream_t s = (cudaStream_t)stream;
    const int np = std::max(16, (int)(2 * N));
    int32_t *dz = nullptr;
    void *bp = nullptr;
    TN_CUDA(cudaMallocAsync((void **)&dz, z.size() * 4, s), "cudaMallocAsync");
    cudaError_t e = cudaMemcpyAsync(dz, z.data(), z.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);        // z is host memory of this call
    if (e == cudaSuccess) e = cudaMallocAsync(&bp, (size_t)np * 2 * K * 2 * m_b, s);
    if (e == cudaSuccess) e = launch_bprep(dtype, B, bp, lk, ln, m_b, np, s);
    if (e == cudaSuccess) {
        TcGemmDesc d;
        d.dtype = dtype;
        d.A = A; d.Bp = bp; d.C = C;
        d.lm = lm; d.ln = ln; d.lk = lk;
        d.batch = T;
        d.batch_a = 1;
        d.batch_b = 1;
        d.np = np;
        d.za = dz;
        d.zb = dz + T;
        d.zc = dz + 2 * T;
        d.depth_a = m_a;
        d.depth_b = m_b;
        if (scheme == TN_GATHER_PADDED && np <= 256) {
            // C_P = A x B_P: each N tile holds R whole B' chunks side by side,
            // so an A tile is loaded once for R places of its padded row
            int R = 1;
            while (R * 2 * np <= 256 && R < m_r) R *= 2;
            d.batch = m_a;
            d.za = nullptr;
            d.gather_r = R;
            d.m_r = m_r;
            d.bn = R * np;
        }
        ScaleRef sr{};
        sr.fixed_exp = scale_exp;
        sr.out_max = out_max;
        e = launch_gemm_tc(d, sr, nullptr, s);
    }
    if (bp) cudaFreeAsync(bp, s);
    cudaFreeAsync(dz, s);
    if (e != cudaSuccess) return cuda_fail(e, "tn_gemm_gather");
    return TN_OK;
}

static int selftest_wait_timeout(void *stream, bool pair) {
    cudaStream_t s = (cudaStream_t)stream;
    // one 128-row tile; pair: one 256 x 256 tile with 128-byte K chunks
    const int lm = pair ? 8 : 7, ln = pair ? 7 : 3, lk = pair ? 5 : 3, np = pair ? 256 : 16;
    void *A = nullptr, *Bp = nullptr, *C = nullptr;
    int32_t *err = nullptr;
    cudaError_t e = cudaMalloc(&A, (size_t)(4 << (lm + lk)));
    if (e == cudaSuccess) e = cudaMalloc(&Bp, (size_t)np * (2 << lk) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&C, (size_t)(4 << (lm + ln)));
    if (e == cudaSuccess) e = cudaMalloc((void **)&err, 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
    int32_t herr = 0;
    if (e == cudaSuccess) {
        TcGemmDesc d;
        d.dtype = TN_F16;
        d.A = A; d.Bp = Bp; d.C = C;
        d.lm = lm; d.ln = ln; d.lk = lk;
        d.batch = 1; d.batch_a = 0; d.batch_b = 0;
        d.np = np;
        d.withhold = 1;
        d.pair = pair ? 1 : 0;
        ScaleRef sr{};
        e = launch_gemm_tc(d, sr, err, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
    }
    cudaFree(A);
    cudaFree(Bp);
    cudaFree(C);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "tn_selftest_wait_timeout");
    if (herr) return fail(TN_ETIMEOUT, "bounded wait gave up as intended; the kernel returned");
    return fail(TN_OK, "no timeout was reported");
}

int tn_selftest_wait_timeout(void *stream) { return selftest_wait_timeout(stream, false); }
int tn_selftest_wait_timeout_pair(void *stream) { return selftest_wait_timeout(stream, true); }

}  // extern "C"
