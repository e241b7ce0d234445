// FP64 norms and inner products of state vectors on the GPU: the reductions the
// precision pattern keeps in FP64 besides the energy and the gradient sums, used for the
// checkpoint norms and for the invariants of Algorithm 1's recurrence (Sec. 2.3: phi and
// lambda are un-applied by the same unitaries, so <lambda_i|phi_{i+1}> stays E and the
// norms of phi and lambda stay constant).
//
// k_norm_dot streams one or two state vectors once (HBM-bound) and writes per-block FP64
// partials of five values,
//   v0 = ||a||^2,  v1 = Re <a|b>,  v2 = Im <a|b>,  v3 = ||b||^2,  v4 = ||a - b||^2
// (<a|b> = sum conj(a_j) b_j; v4 is formed from the differences, not from v0 + v3 - 2 v1,
// so that a small distance is not lost to cancellation),
// to partials[v * nb + block]; launch_reduce_slots sums them over the blocks in a fixed
// order (bit-reproducible).  complex64 products and runs of 16 amplitudes per thread are
// FP32, every run is added to FP64 accumulators; complex128 works in FP64 throughout.
#include "kernels.h"

namespace vqg {

namespace {

constexpr int kNormThreads = 256;

// r += the five values of one 16-byte chunk (two complex64 amplitudes) of a and b
VQG_DEV void acc_chunk(const float4 &x, const float4 &y, float (&r)[5]) {
    const float4 d = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
    r[4] = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, r[4]))));
    r[0] = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, r[0]))));
    r[1] = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, r[1]))));
    r[2] = fmaf(x.x, y.y, fmaf(-x.y, y.x, fmaf(x.z, y.w, fmaf(-x.w, y.z, r[2]))));
    r[3] = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, r[3]))));
}

// HB: a second vector b is given; without it b = a (only ||a||^2 is formed, a is read once)
template <typename T, bool HB>
__global__ void __launch_bounds__(kNormThreads)
    k_norm_dot(const amp_t<T> *__restrict__ a, const amp_t<T> *__restrict__ b, uint64_t n_amp,
               double *__restrict__ partials, int nb) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t first = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if constexpr (sizeof(T) == 4) {
        // 16-byte chunks of two amplitudes (n_amp = 2^n is even); a run is RUN chunks of
        // this thread, summed in FP32 and then added to the FP64 accumulators
        const float4 *__restrict__ a4 = reinterpret_cast<const float4 *>(a);
        const float4 *__restrict__ b4 = reinterpret_cast<const float4 *>(b);
        const uint64_t n_chunk = n_amp / 2;
        constexpr int RUN = 8;
        for (uint64_t c = first; c < n_chunk; c += (uint64_t)RUN * stride) {
            float r[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            float4 x[RUN], y[RUN];
#pragma unroll
            for (int i = 0; i < RUN; ++i) {  // every load of the run in flight first
                const uint64_t ci = c + (uint64_t)i * stride;
                const bool in = ci < n_chunk;
                x[i] = in ? __ldcs(a4 + ci) : make_float4(0.f, 0.f, 0.f, 0.f);
                if constexpr (HB) y[i] = in ? __ldcs(b4 + ci) : make_float4(0.f, 0.f, 0.f, 0.f);
                else y[i] = x[i];
            }
#pragma unroll
            for (int i = 0; i < RUN; ++i) acc_chunk(x[i], y[i], r);
#pragma unroll
            for (int v = 0; v < 5; ++v) acc[v] += (double)r[v];
        }
    } else {
        for (uint64_t j = first; j < n_amp; j += stride) {
            const double2 x = __ldcs(a + j);
            const double2 y = HB ? __ldcs(b + j) : x;
            acc[0] = fma(x.x, x.x, fma(x.y, x.y, acc[0]));
            acc[1] = fma(x.x, y.x, fma(x.y, y.y, acc[1]));
            acc[2] = fma(x.x, y.y, fma(-x.y, y.x, acc[2]));
            acc[3] = fma(y.x, y.x, fma(y.y, y.y, acc[3]));
            const double dx = x.x - y.x, dy = x.y - y.y;
            acc[4] = fma(dx, dx, fma(dy, dy, acc[4]));
        }
    }
    block_reduce_store<5>(acc, partials, nb);
}

}  // namespace

void launch_norm_dot(const void *a, const void *b, int n, bool dbl, double *partials, int nb, cudaStream_t s) {
    const uint64_t n_amp = 1ull << n;
    if (dbl) {
        if (b) k_norm_dot<double, true><<<nb, kNormThreads, 0, s>>>((const double2 *)a, (const double2 *)b, n_amp, partials, nb);
        else k_norm_dot<double, false><<<nb, kNormThreads, 0, s>>>((const double2 *)a, nullptr, n_amp, partials, nb);
    } else {
        if (b) k_norm_dot<float, true><<<nb, kNormThreads, 0, s>>>((const float2 *)a, (const float2 *)b, n_amp, partials, nb);
        else k_norm_dot<float, false><<<nb, kNormThreads, 0, s>>>((const float2 *)a, nullptr, n_amp, partials, nb);
    }
}

}  // namespace vqg
