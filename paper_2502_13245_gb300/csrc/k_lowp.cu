// k_lowp.cu -- low-precision traversal copies of an fp32 index (the precision
// form of the search).  Sec. 5 of the paper traverses float datasets in 8 bits
// and re-ranks so that every reported result is truly within the radius; here
// the traversal copy is BF16 (no scale needed: BF16 keeps fp32's exponent
// range) or FP8-e4m3 with one scale per vector (s = max|x_i| / 448, the e4m3
// maximum), and every membership decision is re-made in exact fp32.
//
// Row layouts (16-byte aligned, zero padded):
//   bf16: d x 2 bytes per row;  fp8: d bytes per row plus, per row, a float2
//   {s, ||x||^2} (the scale and the exact squared norm of the row, used by the
//   squared-L2 form  ||q||^2 - 2 s <q, x8> + ||x||^2).
// The index also records M = max ||x||_2 and M_inf = max |x_i|, which bound
// the traversal error (see slack_coefficients).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <math.h>

#include <algorithm>

#include "rr_common.cuh"

namespace rr {

namespace {

// atomic max on non-negative floats through their bit patterns
__device__ __forceinline__ void atomic_max_pos(float *addr, float v) {
    atomicMax(reinterpret_cast<int *>(addr), __float_as_int(v));
}

// warp per row: bf16 copy, row norms
__global__ void to_bf16_kernel(const float *vec, int64_t n, int d, int in_stride_f, uint16_t *out, int out_stride_h,
                               float *stats) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += nw) {
        const float *x = vec + (size_t)r * in_stride_f;
        uint16_t *o = out + (size_t)r * out_stride_h;
        float ss = 0.f, mx = 0.f;
        for (int i = lane; i < out_stride_h; i += 32) {
            float v = i < d ? x[i] : 0.f;
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            o[i] = *reinterpret_cast<uint16_t *>(&h);
            ss = fmaf(v, v, ss);
            mx = fmaxf(mx, fabsf(v));
        }
        for (int k = 16; k > 0; k >>= 1) {
            ss += __shfl_xor_sync(0xffffffffu, ss, k);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, k));
        }
        if (lane == 0) {
            atomic_max_pos(stats + 0, sqrtf(ss));
            atomic_max_pos(stats + 1, mx);
        }
    }
}

// warp per row: fp8-e4m3 copy with a per-row scale, {s, ||x||^2}
__global__ void to_fp8_kernel(const float *vec, int64_t n, int d, int in_stride_f, uint8_t *out, int out_stride,
                              float2 *info, float *stats) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += nw) {
        const float *x = vec + (size_t)r * in_stride_f;
        float mx = 0.f, ss = 0.f;
        for (int i = lane; i < d; i += 32) {
            mx = fmaxf(mx, fabsf(x[i]));
            ss = fmaf(x[i], x[i], ss);
        }
        for (int k = 16; k > 0; k >>= 1) {
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, k));
            ss += __shfl_xor_sync(0xffffffffu, ss, k);
        }
        const float s = mx > 0.f ? mx / 448.f : 1.f;
        const float inv = 1.f / s;
        uint8_t *o = out + (size_t)r * out_stride;
        for (int i = lane; i < out_stride; i += 32) {
            uint8_t c = 0;
            if (i < d) c = (uint8_t)__nv_cvt_float_to_fp8(x[i] * inv, __NV_SATFINITE, __NV_E4M3);
            o[i] = c;
        }
        if (lane == 0) {
            // the exact squared norm: the squared-L2 form ||q||^2 - 2 s <q,x8> + ||x||^2 then errs
            // only through the dot product
            info[r] = make_float2(s, ss);
            atomic_max_pos(stats + 0, sqrtf(ss));
            atomic_max_pos(stats + 1, mx);
        }
    }
}

}  // namespace

// Build the traversal copy for `prec` once per index (kept until the index is freed).
rr_status ensure_lowp(rr_index *ix, int prec, cudaStream_t st) {
    if (prec == RR_PREC_EXACT) return RR_OK;
    if (ix->dtype != RR_F32) {
        set_error("low-precision traversal needs an fp32 index (8-bit indexes are searched exactly)");
        return RR_EINVAL;
    }
    if (prec != RR_PREC_BF16 && prec != RR_PREC_FP8) {
        set_error("unknown precision %d", prec);
        return RR_EINVAL;
    }
    if (prec == RR_PREC_BF16 && ix->lp_bf16) return RR_OK;
    if (prec == RR_PREC_FP8 && ix->lp_fp8) return RR_OK;
    const int d = ix->d;
    if (!ix->lp_stats) {
        RR_CUDA(cudaMalloc(&ix->lp_stats, 4 * sizeof(float)));
        ix->device_bytes += 16;
    }
    RR_CUDA(cudaMemsetAsync(ix->lp_stats, 0, 2 * sizeof(float), st));
    const int64_t blocks = std::min<int64_t>((ix->n + 7) / 8, 152 * 32);
    if (prec == RR_PREC_BF16) {
        const int stride = (d * 2 + 15) / 16 * 16;
        uint8_t *p = nullptr;
        if (cudaMalloc(&p, (size_t)ix->n * stride) != cudaSuccess) {
            cudaGetLastError();
            set_error("bf16 traversal copy: device allocation failed");
            return RR_ENOMEM;
        }
        to_bf16_kernel<<<(unsigned)blocks, 256, 0, st>>>((const float *)ix->vec, ix->n, d, ix->row_stride / 4,
                                                          (uint16_t *)p, stride / 2, ix->lp_stats);
        RR_CUDA(cudaGetLastError());
        note_launch();
        ix->lp_bf16 = p;
        ix->lp_bf16_stride = stride;
        ix->device_bytes += (int64_t)ix->n * stride;
    } else {
        const int stride = (d + 15) / 16 * 16;
        uint8_t *p = nullptr;
        float2 *info = nullptr;
        if (cudaMalloc(&p, (size_t)ix->n * stride) != cudaSuccess ||
            cudaMalloc(&info, (size_t)ix->n * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            if (p) cudaFree(p);
            set_error("fp8 traversal copy: device allocation failed");
            return RR_ENOMEM;
        }
        to_fp8_kernel<<<(unsigned)blocks, 256, 0, st>>>((const float *)ix->vec, ix->n, d, ix->row_stride / 4, p,
                                                         stride, info, ix->lp_stats);
        RR_CUDA(cudaGetLastError());
        note_launch();
        ix->lp_fp8 = p;
        ix->lp_fp8_info = info;
        ix->lp_fp8_stride = stride;
        ix->device_bytes += (int64_t)ix->n * (stride + 8);
    }
    float h[2];
    RR_CUDA(cudaMemcpyAsync(h, ix->lp_stats, 2 * sizeof(float), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    ix->max_norm = h[0];
    ix->max_abs = h[1];
    return RR_OK;
}

// Absolute slack of the approximate distance: |d - d~| <= A*||q|| + Bq*||q||^2 + C for
// every point x of the index (M = max ||x||, M_inf = max |x_i|, u the relative rounding
// of the traversal format, fp32 accumulation covered by a 1e-5 margin).
//   BF16 (round to nearest, 8 significant bits): |x_i - x~_i| <= 2^-8 |x_i|.
//   FP8-e4m3 with per-row scale s <= M_inf/448: |x_i - x~_i| <= 2^-4 |x_i| + s 2^-10
//   (relative rounding of normals; half the subnormal spacing 2^-9 otherwise).
//   IP:  |<q,x> - <q,x~>| <= sum |q_i||x_i - x~_i| <= u ||q|| M + s 2^-10 ||q||_1,
//        ||q||_1 <= sqrt(d) ||q||.
//   L2, BF16 (sum of (q_i - x~_i)^2):  | ||q-x||^2 - ||q-x~||^2 | <= 2 delta (||q|| + M) +
//        delta^2 with delta = max ||x - x~|| <= u M.
//   L2, FP8 (||q||^2 - 2 s <q,x8> + ||x||^2 with the exact row norm): only the dot
//        product errs, so the bound is twice the IP one.
void slack_coefficients(const rr_index *ix, int prec, float *A, float *Bq, float *C) {
    const double M = ix->max_norm, Minf = ix->max_abs, sd = sqrt((double)ix->d);
    const double u = prec == RR_PREC_BF16 ? 1.0 / 256.0 : 1.0 / 16.0;
    const double sub = prec == RR_PREC_FP8 ? (Minf / 448.0) / 1024.0 : 0.0;
    const double margin = 1e-5;
    if (ix->metric == RR_IP || prec == RR_PREC_FP8) {
        const double k = ix->metric == RR_IP ? 1.0 : 2.0;
        *A = (float)((k * (u * M + sub * sd) + margin * M) * 1.0001);
        *Bq = ix->metric == RR_IP ? 0.f : (float)(margin * 1.0001);
        *C = ix->metric == RR_IP ? 0.f : (float)(margin * M * M * 1.0001);
    } else {
        const double delta = u * M + sub * sd;
        *A = (float)((2.0 * delta + 2.0 * margin * M) * 1.0001);
        *Bq = (float)(margin * 1.0001);
        *C = (float)((2.0 * delta * M + delta * delta + margin * M * M) * 1.0001);
    }
}

}  // namespace rr
