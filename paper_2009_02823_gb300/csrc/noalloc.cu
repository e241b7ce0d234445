// Reverse-sweep steps that allocate nothing.
//
// Some callers cannot allocate device memory while they run this library: code that
// executes while a framework's caching allocator owns the whole device pool, a
// process whose memory is reserved up front and must not grow, or a host thread that
// is forbidden to enter cudaMalloc/cudaFree (which can synchronise the device) in a
// latency-critical loop.  vqg_reverse_noalloc serves them: it runs the fused adjoint
// step on device state vectors the caller owns and keeps its reduction scratch in the
// file-scope array below, which every process that loads the library holds on each
// GPU it touches until the process exits.
//
// Scratch (static, per device):
//   g_noalloc_partials: VQG_NOALLOC_MAX_GATES x 8 x VQG_NOALLOC_BLOCKS doubles (1 MiB),
//                       the per-block partial sums of each gate's four complex sums.
// The gate matrices (U^dagger per gate, D_j = (dU/d slot j) U^dagger per slot) travel as
// kernel parameters, so a call copies nothing from host memory.  Every call overwrites
// the part of the scratch it reads, so nothing needs clearing between calls; calls whose
// work overlaps on the GPU (two streams, two host threads) race on the shared array and
// must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/vqg.h"
#include "common.cuh"

namespace vqg {
int set_error(int status, const char *fmt, ...);
}

namespace {

constexpr int kMaxGates = VQG_NOALLOC_MAX_GATES;
constexpr int kBlocks = VQG_NOALLOC_BLOCKS;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kMaxGates * 8 * kBlocks];

std::mutex g_setup_mutex;
double *g_partials_ptr[kMaxDevices] = {};

// Resolve the device address of the scratch array for the current device, once per
// device: host code may not pass the symbol itself to a kernel (on the host it names a
// stand-in, not device memory).  The cached address belongs to the device's primary
// context; after cudaDeviceReset it is stale.
int setup_device(int dev, double **partials) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess)
            return vqg::set_error(VQG_ERR_CUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        g_partials_ptr[dev] = (double *)p;
    }
    *partials = g_partials_ptr[dev];
    return VQG_OK;
}

// U^dagger of one gate (row-major (re, im) pairs), passed by value.
struct GateMat {
    double m[8];
};

// One adjoint step on pairs of qubit qp (the target for CNOT/CZ): reduce the four
// complex sums o_rc = sum conj(lambda_r) phi_c (phi = phi_{i+1}, lambda = lambda_i),
// then write phi_i = U^dagger phi_{i+1} and U^dagger lambda.  Block partials go to
// partials[v * kBlocks + blockIdx.x], v = 0..7.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_adj_noalloc(amp_t<T> *__restrict__ phi, amp_t<T> *__restrict__ lam, int kind, int q0, int q1,
                  const GateMat mat, uint64_t units, double *__restrict__ partials) {
    const bool ent = kind == K_CNOT || kind == K_CZ;
    const int qp = ent ? q1 : q0;
    const uint64_t bit = 1ull << qp, cbit = 1ull << q0;
    Mat2<T> ud;
    if (!ent) {
#pragma unroll
        for (int k = 0; k < 4; ++k) ud.m[k] = mk<T>((T)mat.m[2 * k], (T)mat.m[2 * k + 1]);
    }
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < units; p += stride) {
        const uint64_t j0 = insert0(p, qp), j1 = j0 | bit;
        amp_t<T> a0 = phi[j0], a1 = phi[j1], l0 = lam[j0], l1 = lam[j1];
        if (!ent) {
            const amp_t<T> o[4] = {cconjmul<T>(l0, a0), cconjmul<T>(l0, a1), cconjmul<T>(l1, a0),
                                   cconjmul<T>(l1, a1)};
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[2 * k] += (double)o[k].x, acc[2 * k + 1] += (double)o[k].y;
            apply2<T>(ud, a0, a1);
            apply2<T>(ud, l0, l1);
        } else if (j0 & cbit) {
            if (kind == K_CNOT) {
                amp_t<T> t = a0; a0 = a1; a1 = t;
                t = l0; l0 = l1; l1 = t;
            } else {
                a1 = mk<T>(-a1.x, -a1.y);
                l1 = mk<T>(-l1.x, -l1.y);
            }
        }
        phi[j0] = a0; phi[j1] = a1;
        lam[j0] = l0; lam[j1] = l1;
    }
    block_reduce_store<8>(acc, partials, kBlocks);
}

// grad[param of slot j of gate k] += 2 Re sum_rc D_rc o_rc.  Warp k sums gate k's eight
// partial columns over the grid (lane l takes blocks l, l+32, ... in order, then a fixed
// shuffle tree), so the result does not depend on timing; thread 0 then adds the slot
// contributions gate by gate in processing order, which keeps the order fixed when
// gates share a parameter.
struct FinishArgs {
    int param[kMaxGates * 3];        // parameter index of slot j of the k-th processed gate, or -1
    double d[kMaxGates * 3 * 8];     // D_j = (dU/d slot j) U^dagger, row-major (re, im) pairs
};

__global__ void __launch_bounds__(32 * kMaxGates)
    k_noalloc_finish(const double *__restrict__ partials, const FinishArgs args, int n_gates, int grid,
                     double *__restrict__ grad) {
    __shared__ double o[kMaxGates][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < n_gates) {
        for (int v = 0; v < 8; ++v) {
            const double *p = partials + ((size_t)warp * 8 + v) * kBlocks;
            double s = 0.0;
            for (int b = lane; b < grid; b += 32) s += p[b];
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
            if (lane == 0) o[warp][v] = s;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int k = 0; k < n_gates; ++k) {
        for (int j = 0; j < 3; ++j) {
            const int param = args.param[3 * k + j];
            if (param < 0) continue;
            const double *d = args.d + 8 * (3 * k + j);
            double acc = 0.0;
            for (int e = 0; e < 4; ++e) acc += d[2 * e] * o[k][2 * e] - d[2 * e + 1] * o[k][2 * e + 1];
            grad[param] += 2.0 * acc;
        }
    }
}

typedef std::complex<double> cd;

void gate_u(int kind, const double *a, cd u[4]) {
    const double c = std::cos(0.5 * a[0]), s = std::sin(0.5 * a[0]);
    const cd I(0.0, 1.0);
    switch (kind) {
    case VQG_RX: u[0] = c; u[1] = -I * s; u[2] = -I * s; u[3] = c; break;
    case VQG_RY: u[0] = c; u[1] = -s; u[2] = s; u[3] = c; break;
    case VQG_RZ: u[0] = std::exp(-0.5 * I * a[0]); u[1] = 0; u[2] = 0; u[3] = std::exp(0.5 * I * a[0]); break;
    default:  // U3
        u[0] = c; u[1] = -std::exp(I * a[2]) * s; u[2] = std::exp(I * a[1]) * s;
        u[3] = std::exp(I * (a[1] + a[2])) * c;
    }
}

// dU/d(slot j)
void gate_du(int kind, int j, const double *a, cd d[4]) {
    const double c = std::cos(0.5 * a[0]), s = std::sin(0.5 * a[0]);
    const cd I(0.0, 1.0);
    cd u[4];
    gate_u(kind, a, u);
    if (kind != VQG_U3) {  // (-i/2) sigma U
        cd sg[4];
        if (kind == VQG_RX) { sg[0] = 0; sg[1] = 1; sg[2] = 1; sg[3] = 0; }
        else if (kind == VQG_RY) { sg[0] = 0; sg[1] = -I; sg[2] = I; sg[3] = 0; }
        else { sg[0] = 1; sg[1] = 0; sg[2] = 0; sg[3] = -1.0; }
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 2; ++cc)
                d[2 * r + cc] = -0.5 * I * (sg[2 * r] * u[cc] + sg[2 * r + 1] * u[2 + cc]);
        return;
    }
    if (j == 0) {
        d[0] = -0.5 * s; d[1] = -std::exp(I * a[2]) * 0.5 * c;
        d[2] = std::exp(I * a[1]) * 0.5 * c; d[3] = -std::exp(I * (a[1] + a[2])) * 0.5 * s;
    } else if (j == 1) {
        d[0] = 0; d[1] = 0; d[2] = I * std::exp(I * a[1]) * s; d[3] = I * std::exp(I * (a[1] + a[2])) * c;
    } else {
        d[0] = 0; d[1] = -I * std::exp(I * a[2]) * s; d[2] = 0; d[3] = I * std::exp(I * (a[1] + a[2])) * c;
    }
}

void put(double *dst, const cd m[4]) {
    for (int e = 0; e < 4; ++e) dst[2 * e] = m[e].real(), dst[2 * e + 1] = m[e].imag();
}

}  // namespace

extern "C" int vqg_reverse_noalloc(int n_qubits, int dtype, const vqg_gate *gates, int n_gates,
                                   const double *theta, int n_params, void *phi, void *lam,
                                   double *grad, void *stream) {
    using namespace vqg;
    if (n_qubits < 1 || n_qubits > 34) return set_error(VQG_ERR_INVALID, "n_qubits=%d outside 1..34", n_qubits);
    if (dtype != VQG_C64 && dtype != VQG_C128) return set_error(VQG_ERR_INVALID, "dtype=%d", dtype);
    if (n_gates < 0 || n_gates > kMaxGates)
        return set_error(VQG_ERR_INVALID, "n_gates=%d: vqg_reverse_noalloc takes at most %d gates per call "
                         "(its static scratch is sized for that); split the sweep into segments", n_gates, kMaxGates);
    if (n_gates == 0) return VQG_OK;
    if (!gates || !phi || !lam || !grad || (!theta && n_params > 0))
        return set_error(VQG_ERR_INVALID, "null pointer");
    // host-side tables on the stack, handed to the kernels as parameters: U^dagger per
    // gate, D_j and the parameter index per slot
    GateMat udag[kMaxGates];
    FinishArgs fin;
    for (int k = 0; k < n_gates; ++k) {
        const vqg_gate &g = gates[n_gates - 1 - k];  // processing order: last gate first
        const bool one = g.kind >= VQG_RX && g.kind <= VQG_U3;
        if (g.kind < VQG_RX || g.kind > VQG_CZ)
            return set_error(VQG_ERR_INVALID, "gate kind %d: vqg_reverse_noalloc takes RX, RY, RZ, U3, CNOT and CZ",
                             g.kind);
        if (g.q0 < 0 || g.q0 >= n_qubits) return set_error(VQG_ERR_INVALID, "qubit %d out of range", g.q0);
        if (!one && (g.q1 < 0 || g.q1 >= n_qubits || g.q1 == g.q0))
            return set_error(VQG_ERR_INVALID, "bad second qubit %d", g.q1);
        const int np = g.kind == VQG_U3 ? 3 : (one ? 1 : 0);
        double a[3] = {0, 0, 0};
        for (int j = 0; j < 3; ++j) {
            fin.param[3 * k + j] = -1;
            if (j < np) {
                if (g.param[j] < 0 || g.param[j] >= n_params)
                    return set_error(VQG_ERR_INVALID, "parameter index %d out of range", g.param[j]);
                a[j] = theta[g.param[j]];
                fin.param[3 * k + j] = g.param[j];
            }
        }
        std::memset(udag[k].m, 0, sizeof(udag[k].m));
        std::memset(fin.d + 24 * k, 0, 24 * sizeof(double));
        if (one) {
            cd u[4], ud[4], du[4], dm[4];
            gate_u(g.kind, a, u);
            ud[0] = std::conj(u[0]); ud[1] = std::conj(u[2]); ud[2] = std::conj(u[1]); ud[3] = std::conj(u[3]);
            put(udag[k].m, ud);
            for (int j = 0; j < np; ++j) {
                gate_du(g.kind, j, a, du);
                for (int r = 0; r < 2; ++r)
                    for (int c = 0; c < 2; ++c) dm[2 * r + c] = du[2 * r] * ud[c] + du[2 * r + 1] * ud[2 + c];
                put(fin.d + 8 * (3 * k + j), dm);
            }
        }
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(VQG_ERR_UNSUPPORTED, "device %d", dev);
    double *partials = nullptr;
    int st = setup_device(dev, &partials);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t pairs = 1ull << (n_qubits - 1);
    const int grid = (int)std::min<uint64_t>(kBlocks, std::max<uint64_t>(1, (pairs + kThreads - 1) / kThreads));
    for (int k = 0; k < n_gates; ++k) {
        const vqg_gate &g = gates[n_gates - 1 - k];
        double *part = partials + (size_t)k * 8 * kBlocks;
        if (dtype == VQG_C64)
            k_adj_noalloc<float><<<grid, kThreads, 0, s>>>((float2 *)phi, (float2 *)lam, g.kind, g.q0, g.q1,
                                                          udag[k], pairs, part);
        else
            k_adj_noalloc<double><<<grid, kThreads, 0, s>>>((double2 *)phi, (double2 *)lam, g.kind, g.q0, g.q1,
                                                           udag[k], pairs, part);
    }
    k_noalloc_finish<<<1, 32 * n_gates, 0, s>>>(partials, fin, n_gates, grid, grad);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "adjoint launch: %s", cudaGetErrorString(e));
    return VQG_OK;
}
