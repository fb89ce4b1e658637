// Low-precision codec for tensors that cross a link (paper Sec. 3.2, Eq. 1,
// Table 1): per group i of a real tensor (complex tensors as their
// interleaved real/imag parts)
//     Q([T]_i) = [T]_i^exp * scale + zero,
//     scale = (q_max - q_min) / (max - min),  zero = (q_min max - q_max min) / (max - min),
// with max/min over the group's transformed values.  Kinds (Table 1):
// half (+-65504, exp 1, whole tensor, not rounded, FP16 codes), int8
// (-128..127, exp 0.2, whole tensor, rounded), int4 (0..15, exp 1, groups of
// `group` values, rounded, two codes per byte, even index in the low nibble).
// x^exp of a negative x is sign(x)|x|^exp; rounding is to nearest even, then
// clamped; a group of equal values gets scale 1 and zero q_min - value.
// Every operation that decides a code is one rounded FP32 operation (no
// contraction into FMA), in the order the formulas are written.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"
#include "plan.h"

namespace tn {
namespace {

struct KindParams {
    float q_min, q_max, exp;
    int rounded;
};

__host__ __device__ inline KindParams kind_params(int kind) {
    switch (kind) {
        case TN_CODEC_INT8: return {-128.0f, 127.0f, 0.2f, 1};
        case TN_CODEC_INT4: return {0.0f, 15.0f, 1.0f, 1};
        default: return {-65504.0f, 65504.0f, 1.0f, 0};
    }
}

__device__ __forceinline__ float transform(float x, float exp) {
    if (exp == 1.0f) return x;
    const float a = powf(fabsf(x), exp);
    return x < 0.0f ? -a : (x > 0.0f ? a : 0.0f);
}

__device__ __forceinline__ void scale_zero(float lo, float hi, const KindParams &k, float &scale,
                                           float &zero) {
    const float span = __fsub_rn(hi, lo);
    if (span == 0.0f) {
        scale = 1.0f;
        zero = __fsub_rn(k.q_min, lo);
    } else {
        scale = __fdiv_rn(k.q_max - k.q_min, span);
        zero = __fdiv_rn(__fsub_rn(__fmul_rn(k.q_min, hi), __fmul_rn(k.q_max, lo)), span);
    }
}

__device__ __forceinline__ float code_value(float y, float scale, float zero, const KindParams &k) {
    const float v = __fadd_rn(__fmul_rn(y, scale), zero);
    if (!k.rounded) return v;
    return fminf(fmaxf(rintf(v), k.q_min), k.q_max);
}

// ---- whole-tensor kinds: block min/max partials, then one block finishes
__global__ void minmax_partial_kernel(const float *__restrict__ x, int64_t n, float exp, float2 *part) {
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float y = transform(x[i], exp);
        lo = fminf(lo, y);
        hi = fmaxf(hi, y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ float2 w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = make_float2(lo, hi);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            lo = fminf(lo, w[i].x);
            hi = fmaxf(hi, w[i].y);
        }
        part[blockIdx.x] = make_float2(lo, hi);
    }
}

__global__ void minmax_final_kernel(const float2 *part, int n_part, int kind, float *scale, float *zero) {
    if (threadIdx.x != 0) return;
    float lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < n_part; ++i) {
        lo = fminf(lo, part[i].x);
        hi = fmaxf(hi, part[i].y);
    }
    const KindParams k = kind_params(kind);
    scale_zero(lo, hi, k, scale[0], zero[0]);
}

template <int KIND>
__global__ void encode_whole_kernel(const float *__restrict__ x, int64_t n, const float *scale,
                                    const float *zero, void *codes) {
    const KindParams k = kind_params(KIND);
    const float s = scale[0], z = zero[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = code_value(transform(x[i], k.exp), s, z, k);
        if constexpr (KIND == TN_CODEC_HALF)
            reinterpret_cast<__half *>(codes)[i] = __float2half_rn(v);
        else
            reinterpret_cast<int8_t *>(codes)[i] = (int8_t)(int)v;
    }
}

// ---- int4 groups: one warp per group, 4 values per lane per pass
__global__ void encode_int4_kernel(const float *__restrict__ x, int64_t n_groups, int group,
                                   uint8_t *__restrict__ codes, float *scale, float *zero) {
    const KindParams k = kind_params(TN_CODEC_INT4);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n_groups; g += warps) {
        const float4 *src = reinterpret_cast<const float4 *>(x + g * group);
        float lo = INFINITY, hi = -INFINITY;
        float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f);    // groups of 128: one float4 per lane, kept
        if (group == 128) {
            v0 = src[lane];
            lo = fminf(fminf(v0.x, v0.y), fminf(v0.z, v0.w));
            hi = fmaxf(fmaxf(v0.x, v0.y), fmaxf(v0.z, v0.w));
        }
        for (int i = lane; group != 128 && i < group / 4; i += 32) {
            const float4 v = src[i];
            lo = fminf(fminf(lo, v.x), fminf(v.y, fminf(v.z, v.w)));
            hi = fmaxf(fmaxf(hi, v.x), fmaxf(v.y, fmaxf(v.z, v.w)));
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        float s, z;
        scale_zero(lo, hi, k, s, z);
        if (lane == 0) {
            scale[g] = s;
            zero[g] = z;
        }
        uint16_t *dst = reinterpret_cast<uint16_t *>(codes + g * (group / 2));
        for (int i = lane; i < group / 4; i += 32) {
            const float4 v = group == 128 ? v0 : src[i];
            const unsigned c0 = (unsigned)code_value(v.x, s, z, k), c1 = (unsigned)code_value(v.y, s, z, k);
            const unsigned c2 = (unsigned)code_value(v.z, s, z, k), c3 = (unsigned)code_value(v.w, s, z, k);
            dst[i] = (uint16_t)(c0 | (c1 << 4) | (c2 << 8) | (c3 << 12));
        }
    }
}

template <int KIND>
__global__ void decode_kernel(const void *__restrict__ codes, const float *scale, const float *zero,
                              int64_t n, int group, float *__restrict__ x) {
    const KindParams k = kind_params(KIND);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float q;
        int64_t g = 0;
        if constexpr (KIND == TN_CODEC_HALF) {
            q = __half2float(reinterpret_cast<const __half *>(codes)[i]);
        } else if constexpr (KIND == TN_CODEC_INT8) {
            q = (float)reinterpret_cast<const int8_t *>(codes)[i];
        } else {
            const uint8_t b = reinterpret_cast<const uint8_t *>(codes)[i >> 1];
            q = (float)((i & 1) ? (b >> 4) : (b & 15));
            g = i / group;
        }
        const float y = __fdiv_rn(__fsub_rn(q, zero[g]), scale[g]);
        x[i] = k.exp == 1.0f ? y : (y < 0.0f ? -powf(-y, 1.0f / k.exp) : powf(y, 1.0f / k.exp));
    }
}

int grid_for(int64_t n, int threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, (int64_t)tc_num_sms() * 8));
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

int tn_encode(int32_t kind, const float *x, int64_t n, int32_t group, void *codes, float *scale, float *zero,
              void *stream) {
    if (!x || !codes || !scale || !zero) return record_error(TN_EINVAL, "NULL argument");
    if (n < 1) return record_error(TN_EINVAL, "n must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (kind == TN_CODEC_INT4) {
        if (group < 128 || group > 65536 || (group & (group - 1)) || n % group)
            return record_error(TN_EINVAL, "int4 groups: a power of two in 128..65536 dividing n");
        const int64_t ng = n / group;
        const int threads = 256;
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((ng + 7) / 8, (int64_t)tc_num_sms() * 16));
        encode_int4_kernel<<<blocks, threads, 0, s>>>(x, ng, group, (uint8_t *)codes, scale, zero);
        e = cudaGetLastError();
    } else if (kind == TN_CODEC_HALF || kind == TN_CODEC_INT8) {
        if (group != 0) return record_error(TN_EINVAL, "half and int8 use one group (group = 0)");
        const int threads = 256;
        const int blocks = grid_for(n, threads);
        float2 *part = nullptr;
        e = cudaMallocAsync((void **)&part, sizeof(float2) * blocks, s);
        if (e == cudaSuccess) {
            minmax_partial_kernel<<<blocks, threads, 0, s>>>(x, n, kind_params(kind).exp, part);
            minmax_final_kernel<<<1, 32, 0, s>>>(part, blocks, kind, scale, zero);
            if (kind == TN_CODEC_HALF)
                encode_whole_kernel<TN_CODEC_HALF><<<blocks, threads, 0, s>>>(x, n, scale, zero, codes);
            else
                encode_whole_kernel<TN_CODEC_INT8><<<blocks, threads, 0, s>>>(x, n, scale, zero, codes);
            e = cudaGetLastError();
            cudaFreeAsync(part, s);
        }
    } else {
        return record_error(TN_EINVAL, "unknown codec kind");
    }
    if (e != cudaSuccess) return record_error(TN_ECUDA, std::string("tn_encode: ") + cudaGetErrorString(e));
    return TN_OK;
}

int tn_decode(int32_t kind, const void *codes, const float *scale, const float *zero, int64_t n, int32_t group,
              float *x, void *stream) {
    if (!x || !codes || !scale || !zero) return record_error(TN_EINVAL, "NULL argument");
    if (n < 1) return record_error(TN_EINVAL, "n must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256;
    const int blocks = grid_for(n, threads);
    if (kind == TN_CODEC_INT4) {
        if (group < 128 || group > 65536 || (group & (group - 1)) || n % group)
            return record_error(TN_EINVAL, "int4 groups: a power of two in 128..65536 dividing n");
        decode_kernel<TN_CODEC_INT4><<<blocks, threads, 0, s>>>(codes, scale, zero, n, group, x);
    } else if (kind == TN_CODEC_INT8) {
        decode_kernel<TN_CODEC_INT8><<<blocks, threads, 0, s>>>(codes, scale, zero, n, 0, x);
    } else if (kind == TN_CODEC_HALF) {
        decode_kernel<TN_CODEC_HALF><<<blocks, threads, 0, s>>>(codes, scale, zero, n, 0, x);
    } else {
        return record_error(TN_EINVAL, "unknown codec kind");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_error(TN_ECUDA, std::string("tn_decode: ") + cudaGetErrorString(e));
    return TN_OK;
}

}  // extern "C"
