// Device-side helpers shared by the kernels of the GB300 library: complex
// arithmetic on interleaved (re, im) amplitudes, bit insertion for pair
// enumeration, and deterministic FP64 block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define VQG_DEV __device__ __forceinline__

// ----------------------------------------------------------------- amplitude types
template <typename T> struct Amp;
template <> struct Amp<float> { using type = float2; };
template <> struct Amp<double> { using type = double2; };
template <typename T> using amp_t = typename Amp<T>::type;

template <typename T> VQG_DEV amp_t<T> mk(T re, T im) { amp_t<T> r; r.x = re; r.y = im; return r; }
template <typename T> VQG_DEV amp_t<T> cadd(amp_t<T> a, amp_t<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> VQG_DEV amp_t<T> cmul(amp_t<T> a, amp_t<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a*b + c
template <typename T> VQG_DEV amp_t<T> cfma(amp_t<T> a, amp_t<T> b, amp_t<T> c) {
    return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// conj(a) * b
template <typename T> VQG_DEV amp_t<T> cconjmul(amp_t<T> a, amp_t<T> b) {
    return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// 2x2 complex matrix in registers, row-major: m[0]=m00, m[1]=m01, m[2]=m10, m[3]=m11.
template <typename T> struct Mat2 { amp_t<T> m[4]; };

// Load U from the FP64 gate table (8 doubles, row-major re/im) rounded to T.
template <typename T> VQG_DEV Mat2<T> load_mat(const double *__restrict__ g) {
    Mat2<T> r;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.m[k] = mk<T>((T)__ldg(g + 2 * k), (T)__ldg(g + 2 * k + 1));
    return r;
}
// U^dagger from the table.
template <typename T> VQG_DEV Mat2<T> load_mat_dagger(const double *__restrict__ g) {
    Mat2<T> u = load_mat<T>(g), r;
    r.m[0] = mk<T>(u.m[0].x, -u.m[0].y);
    r.m[1] = mk<T>(u.m[2].x, -u.m[2].y);
    r.m[2] = mk<T>(u.m[1].x, -u.m[1].y);
    r.m[3] = mk<T>(u.m[3].x, -u.m[3].y);
    return r;
}

template <typename T> VQG_DEV void apply2(const Mat2<T> &u, amp_t<T> &a0, amp_t<T> &a1) {
    amp_t<T> b0 = cfma<T>(u.m[1], a1, cmul<T>(u.m[0], a0));
    amp_t<T> b1 = cfma<T>(u.m[3], a1, cmul<T>(u.m[2], a0));
    a0 = b0;
    a1 = b1;
}

// ----------------------------------------------------------------- index helpers
// Insert a zero bit at position b of x (the pair enumeration of a one-qubit gate).
VQG_DEV uint64_t insert0(uint64_t x, int b) {
    uint64_t lo = x & ((1ull << b) - 1ull);
    return ((x >> b) << (b + 1)) | lo;
}
// Insert zero bits at positions lo < hi.
VQG_DEV uint64_t insert00(uint64_t x, int lo, int hi) { return insert0(insert0(x, lo), hi); }

// ----------------------------------------------------------------- reductions
VQG_DEV double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block reduction of NV FP64 values per thread; thread 0 writes
// partials[v * nb + blockIdx.x].  Requires blockDim.x a multiple of 32, <= 1024.
template <int NV>
VQG_DEV void block_reduce_store(const double (&acc)[NV], double *__restrict__ partials, int nb) {
    __shared__ double red[32][NV > 0 ? NV : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double s = warp_sum(acc[v]);
        if (lane == 0) red[warp][v] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double s = lane < nw ? red[lane][v] : 0.0;
            s = warp_sum(s);
            if (lane == 0) partials[(size_t)v * nb + blockIdx.x] = s;
        }
    }
}

// Gate kinds (mirror of vqg_gate_kind; the ABI header is C, kernels use these).
enum : int {
    K_RX = 0, K_RY = 1, K_RZ = 2, K_U3 = 3, K_CNOT = 4, K_CZ = 5,
    K_CRX = 6, K_CRY = 7, K_CRZ = 8, K_PHASE = 9, K_CPHASE = 10
};

// Controlled kinds with a parameter: their 2x2 matrix acts on q1 where q0 is 1.
__host__ __device__ constexpr bool is_controlled_param(int kind) {
    return (kind >= K_CRX && kind <= K_CRZ) || kind == K_CPHASE;
}
// Kinds with a parameter-dependent 2x2 matrix in the gate table.
__host__ __device__ constexpr bool has_matrix(int kind) { return kind <= K_U3 || kind >= K_CRX; }
// Parameters of a kind (parameter slots used).
__host__ __device__ constexpr int params_of(int kind) {
    return kind == K_U3 ? 3 : (has_matrix(kind) ? 1 : 0);
}

// Number of reduction values a gate contributes in the reverse sweep:
// rotations (controlled or not) reduce Im<lambda|P sigma|phi> and phase gates
// -2 Im<lambda|P|1><1|phi> (1 value; P projects onto control = 1, App. A); a general
// one-qubit gate reduces the four complex sums o_rc = sum conj(lambda_r) phi_c
// (8 values) that its derivative matrices are contracted with afterwards; entanglers
// reduce nothing.
__host__ __device__ constexpr int reduce_values_of(int kind) {
    return kind == K_U3 ? 8 : (has_matrix(kind) ? 1 : 0);
}

// One Pauli term of an x-group: w = coef * i^{popcount(x & z)}.
struct PauliTerm {
    uint64_t z;
    double wr, wi;
};
