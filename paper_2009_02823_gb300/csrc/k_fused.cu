// Tile-fused sweeps (the gate-fusion scheme of the GB300 design; the paper's
// algorithm only needs "apply gate" primitives, Sec. 2.1, and leaves their fusion to
// the simulator).
//
//   k_fused_fwd : one forward pass -- every tile of 2^K amplitudes is read from HBM once,
//                 a run of gates is applied in shared memory / registers, and the tile
//                 is written once (Algorithm 1, line 2, many gates per state traversal).
//   k_fused_rev : one reverse pass -- phi and lambda tiles are read once, and for each
//                 gate of the run in reverse order the kernel reduces the gradient sums
//                 from (phi_{i+1}, lambda_i) and un-applies U_i^dagger to both
//                 (Algorithm 1, lines 6-11, with App. A's dR = -(i/2) sigma R so that
//                 mu = dU phi is never formed; App. B.1 for U3).
//   k_fused_ham : one Hamiltonian pass -- the Pauli groups whose flip mask lies inside
//                 the tile, lambda (+)= sum_g f_g(j^x) psi[j^x], with E = Re<psi|lambda>.
//
// Reduction precision (complex64 amplitudes): products in FP32, per-thread runs of at
// most 16 terms in FP32, the 32-lane warp tree in FP32, then every warp sum is added
// into an FP64 accumulator (shared memory), and block / grid levels are FP64.
#include <type_traits>

#include "fused.h"
#include "kernels.h"

namespace vqg {

template <typename T> struct FT;
template <> struct FT<float> { static constexpr int L = 4, AB = 8; };
template <> struct FT<double> { static constexpr int L = 3, AB = 16; };

template <typename T> VQG_DEV T shfl(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

template <typename T> VQG_DEV T warp_tree(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl(v, o);
    return v;
}

// Reduce 8 values over the warp with 9 shuffles; returns the total of value index
// ((lane>>4)&1)*4 + ((lane>>3)&1)*2 + ((lane>>2)&1), identical on the 4 lanes sharing
// those bits.
template <typename T> VQG_DEV T warp_reduce8(const T (&v)[8]) {
    const int lane = threadIdx.x & 31;
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    T k4[4], k2[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) k4[i] = (h4 ? v[i + 4] : v[i]) + shfl(h4 ? v[i] : v[i + 4], 16);
#pragma unroll
    for (int i = 0; i < 2; ++i) k2[i] = (h3 ? k4[i + 2] : k4[i]) + shfl(h3 ? k4[i] : k4[i + 2], 8);
    T k1 = (h2 ? k2[1] : k2[0]) + shfl(h2 ? k2[0] : k2[1], 4);
    k1 += shfl(k1, 2);
    k1 += shfl(k1, 1);
    return k1;
}

template <int R, typename F> VQG_DEV void with_k(int k, F &&f) {
    switch (k) {
    case 0: f(std::integral_constant<int, 0>{}); break;
    case 1: if constexpr (R > 1) f(std::integral_constant<int, 1>{}); break;
    case 2: if constexpr (R > 2) f(std::integral_constant<int, 2>{}); break;
    case 3: if constexpr (R > 3) f(std::integral_constant<int, 3>{}); break;
    case 4: if constexpr (R > 4) f(std::integral_constant<int, 4>{}); break;
    default: break;
    }
}

template <typename T> VQG_DEV amp_t<T> neg(amp_t<T> a) { return mk<T>(-a.x, -a.y); }

// ------------------------------------------------------------------ gate ops (forward)
template <int KB, int NA, typename T>
VQG_DEV void op_ry(amp_t<T> (&a)[NA], T c, T s) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        const int j1 = j | (1 << KB);
        const amp_t<T> x = a[j], y = a[j1];
        a[j] = mk<T>(c * x.x - s * y.x, c * x.y - s * y.y);
        a[j1] = mk<T>(s * x.x + c * y.x, s * x.y + c * y.y);
    }
}

template <int KB, int NA, typename T>
VQG_DEV void op_gen(amp_t<T> (&a)[NA], const Mat2<T> &u) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        apply2<T>(u, a[j], a[j | (1 << KB)]);
    }
}

template <int KB, int NA, typename T>
VQG_DEV void op_rzr(amp_t<T> (&a)[NA], amp_t<T> p0, amp_t<T> p1) {
#pragma unroll
    for (int j = 0; j < NA; ++j) a[j] = cmul<T>((j & (1 << KB)) ? p1 : p0, a[j]);
}

template <int NA, typename T>
VQG_DEV void op_rzt(amp_t<T> (&a)[NA], amp_t<T> p) {
#pragma unroll
    for (int j = 0; j < NA; ++j) a[j] = cmul<T>(p, a[j]);
}

// negate a[j] where (j & need) == need, if thr_ok
template <int NA, typename T>
VQG_DEV void op_cz(amp_t<T> (&a)[NA], uint32_t need, bool thr_ok) {
    if (!thr_ok) return;
#pragma unroll
    for (int j = 0; j < NA; ++j)
        if ((j & need) == need) a[j] = neg<T>(a[j]);
}

template <int KB, int NA, typename T>
VQG_DEV void op_cnot(amp_t<T> (&a)[NA], uint32_t rc, bool thr_c) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        const bool c = rc ? ((j & rc) != 0) : thr_c;
        if (c) {
            const amp_t<T> t = a[j];
            a[j] = a[j | (1 << KB)];
            a[j | (1 << KB)] = t;
        }
    }
}

template <typename T> VQG_DEV Mat2<T> mat_of(const T *__restrict__ m) {
    Mat2<T> u;
#pragma unroll
    for (int k = 0; k < 4; ++k) u.m[k] = mk<T>(m[2 * k], m[2 * k + 1]);
    return u;
}

template <typename T> VQG_DEV Mat2<T> dagger(const Mat2<T> &u) {
    Mat2<T> r;
    r.m[0] = mk<T>(u.m[0].x, -u.m[0].y);
    r.m[1] = mk<T>(u.m[2].x, -u.m[2].y);
    r.m[2] = mk<T>(u.m[1].x, -u.m[1].y);
    r.m[3] = mk<T>(u.m[3].x, -u.m[3].y);
    return r;
}

template <int R, int NA, typename T>
VQG_DEV void apply_fwd_op(amp_t<T> (&a)[NA], const FOp &op, uint64_t gb, const T *__restrict__ mats) {
    const T *m = mats + 8 * (size_t)op.gate;
    switch (op.type) {
    case OP_RY: {
        const T c = m[0], s = m[4];
        with_k<R>(op.k, [&](auto kb) { op_ry<decltype(kb)::value, NA, T>(a, c, s); });
        break;
    }
    case OP_RX:
    case OP_U3: {
        const Mat2<T> u = mat_of<T>(m);
        with_k<R>(op.k, [&](auto kb) { op_gen<decltype(kb)::value, NA, T>(a, u); });
        break;
    }
    case OP_RZ_REG: {
        const amp_t<T> p0 = mk<T>(m[0], m[1]), p1 = mk<T>(m[6], m[7]);
        with_k<R>(op.k, [&](auto kb) { op_rzr<decltype(kb)::value, NA, T>(a, p0, p1); });
        break;
    }
    case OP_RZ_THR: {
        const bool b = (gb & op.g0) != 0;
        op_rzt<NA, T>(a, b ? mk<T>(m[6], m[7]) : mk<T>(m[0], m[1]));
        break;
    }
    case OP_CZ: {
        const bool ok = (op.rm0 || (gb & op.g0)) && (op.rm1 || (gb & op.g1));
        op_cz<NA, T>(a, op.rm0 | op.rm1, ok);
        break;
    }
    case OP_CNOT: {
        const bool c = (gb & op.g0) != 0;
        with_k<R>(op.k, [&](auto kb) { op_cnot<decltype(kb)::value, NA, T>(a, op.rm0, c); });
        break;
    }
    default:
        break;
    }
}

// ------------------------------------------------------------------ gate ops (reverse)
// Each returns the thread's partial of the gate's reduction value(s) computed from
// (phi_{i+1} = a, lambda_i = l) before un-applying U^dagger to both.
template <int KB, int NA, typename T>
VQG_DEV T rev_ry(amp_t<T> (&a)[NA], amp_t<T> (&l)[NA], T c, T s) {
    T v = 0;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        const int j1 = j | (1 << KB);
        const amp_t<T> a0 = a[j], a1 = a[j1], l0 = l[j], l1 = l[j1];
        // Im <lambda| Y |phi> over the pair: Re(conj(l1) a0) - Re(conj(l0) a1)
        v += (l1.x * a0.x + l1.y * a0.y) - (l0.x * a1.x + l0.y * a1.y);
        // RY^dagger = [[c, s], [-s, c]]
        a[j] = mk<T>(c * a0.x + s * a1.x, c * a0.y + s * a1.y);
        a[j1] = mk<T>(c * a1.x - s * a0.x, c * a1.y - s * a0.y);
        l[j] = mk<T>(c * l0.x + s * l1.x, c * l0.y + s * l1.y);
        l[j1] = mk<T>(c * l1.x - s * l0.x, c * l1.y - s * l0.y);
    }
    return v;
}

template <int KB, int NA, typename T>
VQG_DEV T rev_rx(amp_t<T> (&a)[NA], amp_t<T> (&l)[NA], const Mat2<T> &ud) {
    T v = 0;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        const int j1 = j | (1 << KB);
        const amp_t<T> a0 = a[j], a1 = a[j1], l0 = l[j], l1 = l[j1];
        // Im <lambda| X |phi>: Im(conj(l0) a1) + Im(conj(l1) a0)
        v += (l0.x * a1.y - l0.y * a1.x) + (l1.x * a0.y - l1.y * a0.x);
        apply2<T>(ud, a[j], a[j1]);
        apply2<T>(ud, l[j], l[j1]);
    }
    return v;
}

template <int KB, int NA, typename T>
VQG_DEV void rev_u3(amp_t<T> (&a)[NA], amp_t<T> (&l)[NA], const Mat2<T> &ud, T (&v)[8]) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        const int j1 = j | (1 << KB);
        const amp_t<T> a0 = a[j], a1 = a[j1], l0 = l[j], l1 = l[j1];
        const amp_t<T> o00 = cconjmul<T>(l0, a0), o01 = cconjmul<T>(l0, a1);
        const amp_t<T> o10 = cconjmul<T>(l1, a0), o11 = cconjmul<T>(l1, a1);
        v[0] += o00.x; v[1] += o00.y; v[2] += o01.x; v[3] += o01.y;
        v[4] += o10.x; v[5] += o10.y; v[6] += o11.x; v[7] += o11.y;
        apply2<T>(ud, a[j], a[j1]);
        apply2<T>(ud, l[j], l[j1]);
    }
}

// Im <lambda| Z |phi> with Z on a register bit, then the conjugate phases.
template <int KB, int NA, typename T>
VQG_DEV T rev_rzr(amp_t<T> (&a)[NA], amp_t<T> (&l)[NA], amp_t<T> q0, amp_t<T> q1) {
    T v = 0;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const T im = l[j].x * a[j].y - l[j].y * a[j].x;
        v += (j & (1 << KB)) ? -im : im;
        const amp_t<T> q = (j & (1 << KB)) ? q1 : q0;
        a[j] = cmul<T>(q, a[j]);
        l[j] = cmul<T>(q, l[j]);
    }
    return v;
}

template <int NA, typename T>
VQG_DEV T rev_rzt(amp_t<T> (&a)[NA], amp_t<T> (&l)[NA], amp_t<T> q, bool minus) {
    T v = 0;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        v += l[j].x * a[j].y - l[j].y * a[j].x;
        a[j] = cmul<T>(q, a[j]);
        l[j] = cmul<T>(q, l[j]);
    }
    return minus ? -v : v;
}

// ------------------------------------------------------------------ tile I/O
template <typename T, int K>
struct TileIO {
    static constexpr int L = FT<T>::L, AB = FT<T>::AB;
    static constexpr int TILE = 1 << K, ROWS = 1 << (K - L);
    static constexpr int CA = 16 / AB;          // amplitudes per 16-byte chunk
    static constexpr int CPR = (1 << L) / CA;   // chunks per 128-byte row
    static constexpr int CHUNKS = TILE / CA;

    static VQG_DEV void load(amp_t<T> *tile, const amp_t<T> *__restrict__ src, uint64_t base,
                             const uint64_t *row_off, int tid, int nt) {
        for (int c = tid; c < CHUNKS; c += nt) {
            const int row = c / CPR, col = c % CPR;
            const uint32_t t = (uint32_t)(row << L) | (uint32_t)(col * CA);
            const float4 v = __ldcs(reinterpret_cast<const float4 *>(src + (base | row_off[row]) + col * CA));
            put_chunk(tile, t, v);
        }
    }
    static VQG_DEV void zero(amp_t<T> *tile, uint64_t base, int tid, int nt) {
        for (int c = tid; c < CHUNKS; c += nt) put_chunk(tile, (uint32_t)(c * CA), make_float4(0.f, 0.f, 0.f, 0.f));
        if (base == 0 && tid == 0) tile[swz<AB>(0)] = mk<T>((T)1, (T)0);
    }
    // A 16-byte chunk (two complex64 or one complex128 amplitudes starting at tile-local
    // index t) to / from shared memory.  The complex64 swizzle may separate the two
    // amplitudes (it folds higher bits into bit 0), so each goes to its own 8-byte slot.
    static VQG_DEV void put_chunk(amp_t<T> *tile, uint32_t t, float4 v) {
        if constexpr (AB == 8) {
            tile[swz<AB>(t)] = mk<T>(v.x, v.y);
            tile[swz<AB>(t + 1)] = mk<T>(v.z, v.w);
        } else {
            *reinterpret_cast<float4 *>(tile + swz<AB>(t)) = v;
        }
    }
    static VQG_DEV float4 get_chunk(const amp_t<T> *tile, uint32_t t) {
        if constexpr (AB == 8) {
            const amp_t<T> a = tile[swz<AB>(t)], b = tile[swz<AB>(t + 1)];
            return make_float4(a.x, a.y, b.x, b.y);
        } else {
            return *reinterpret_cast<const float4 *>(tile + swz<AB>(t));
        }
    }
    static VQG_DEV void store(const amp_t<T> *tile, amp_t<T> *__restrict__ dst, uint64_t base,
                              const uint64_t *row_off, int tid, int nt) {
        for (int c = tid; c < CHUNKS; c += nt) {
            const int row = c / CPR, col = c % CPR;
            const uint32_t t = (uint32_t)(row << L) | (uint32_t)(col * CA);
            __stcs(reinterpret_cast<float4 *>(dst + (base | row_off[row]) + col * CA), get_chunk(tile, t));
        }
    }
};

VQG_DEV uint64_t tile_base(uint64_t tile, const int32_t *nontile, int n_nontile) {
    uint64_t b = 0;
    for (int i = 0; i < n_nontile; ++i) b |= ((tile >> i) & 1ull) << nontile[i];
    return b;
}

// Shared-memory prologue common to the sweep kernels: the pass's stages and ops and
// the row-offset table.
template <typename T, int K>
VQG_DEV void load_pass(const FPass &P, int stage0, int n_stage, const FStage *__restrict__ stages,
                       const FOp *__restrict__ ops, FStage *sst, FOp *sop, uint64_t *row_off, int tid, int nt) {
    constexpr int L = FT<T>::L, ROWS = 1 << (K - L);
    const int op0 = n_stage ? stages[stage0].op0 : 0;
    const int op_end = n_stage ? stages[stage0 + n_stage - 1].op0 + stages[stage0 + n_stage - 1].n_op : 0;
    {
        const int words = n_stage * (int)(sizeof(FStage) / 4);
        const uint32_t *s = reinterpret_cast<const uint32_t *>(stages + stage0);
        uint32_t *d = reinterpret_cast<uint32_t *>(sst);
        for (int i = tid; i < words; i += nt) d[i] = s[i];
    }
    {
        const int words = (op_end - op0) * (int)(sizeof(FOp) / 4);
        const uint32_t *s = reinterpret_cast<const uint32_t *>(ops + op0);
        uint32_t *d = reinterpret_cast<uint32_t *>(sop);
        for (int i = tid; i < words; i += nt) d[i] = s[i];
    }
    for (int r = tid; r < ROWS; r += nt) {
        uint64_t off = 0;
        for (int i = 0; i < K - L; ++i)
            if ((r >> i) & 1) off |= 1ull << P.high[i];
        row_off[r] = off;
    }
}

template <typename T, int K, int R>
struct FwdCfg {
    static constexpr int NT = 1 << (K - R);
    static constexpr size_t smem() {
        return (size_t)(1 << K) * FT<T>::AB + sizeof(uint64_t) * (1 << (K - FT<T>::L)) +
               sizeof(FStage) * kMaxPassStages + sizeof(FOp) * kMaxPassOps;
    }
};

// ------------------------------------------------------------------ forward pass
template <typename T, int K, int R>
__global__ void __launch_bounds__(1 << (K - R))
    k_fused_fwd(const amp_t<T> *__restrict__ src, amp_t<T> *__restrict__ dst,
                const FPass *__restrict__ passes, int pi, const FStage *__restrict__ stages,
                const FOp *__restrict__ ops, const T *__restrict__ mats, uint64_t n_tiles) {
    using A = amp_t<T>;
    using IO = TileIO<T, K>;
    constexpr int AB = FT<T>::AB, NT = 1 << (K - R), NA = 1 << R;
    extern __shared__ __align__(16) unsigned char smem[];
    A *tile = reinterpret_cast<A *>(smem);
    uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + (size_t)(1 << K) * AB);
    FStage *sst = reinterpret_cast<FStage *>(row_off + IO::ROWS);
    FOp *sop = reinterpret_cast<FOp *>(sst + kMaxPassStages);
    const FPass &P = passes[pi];
    const int tid = threadIdx.x;
    const int n_stage = P.n_stage;
    load_pass<T, K>(P, P.stage0, n_stage, stages, ops, sst, sop, row_off, tid, NT);
    const int op_base = n_stage ? stages[P.stage0].op0 : 0;
    const int n_nontile = P.n_nontile;
    const bool from_zero = P.from_zero;
    __syncthreads();
    for (uint64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const uint64_t base = tile_base(ti, P.nontile, n_nontile);
        if (from_zero) IO::zero(tile, base, tid, NT);
        else IO::load(tile, src, base, row_off, tid, NT);
        __syncthreads();
        for (int s = 0; s < n_stage; ++s) {
            const FStage &st = sst[s];
            uint32_t sb = 0;
            uint64_t gb = base;
#pragma unroll
            for (int b = 0; b < K - R; ++b)
                if ((tid >> b) & 1) sb ^= st.thr_sw[b], gb |= st.thr_g[b];
            uint32_t w[R];
#pragma unroll
            for (int k = 0; k < R; ++k) w[k] = st.reg_sw[k];
            A a[NA];
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                uint32_t ad = sb;
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if ((j >> k) & 1) ad ^= w[k];
                a[j] = tile[ad];
            }
            const int o_end = st.op0 - op_base + st.n_op;
            for (int o = st.op0 - op_base; o < o_end; ++o) apply_fwd_op<R, NA, T>(a, sop[o], gb, mats);
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                uint32_t ad = sb;
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if ((j >> k) & 1) ad ^= w[k];
                tile[ad] = a[j];
            }
            __syncthreads();
        }
        IO::store(tile, dst, base, row_off, tid, NT);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ reverse pass
template <typename T, int K, int R>
struct RevCfg {
    static constexpr int NT = 1 << (K - R), NW = NT / 32;
    static constexpr size_t smem() {
        return 2 * (size_t)(1 << K) * FT<T>::AB + sizeof(uint64_t) * (1 << (K - FT<T>::L)) +
               sizeof(FStage) * kMaxPassStages + sizeof(FOp) * kMaxPassOps +
               sizeof(double) * (size_t)NW * kMaxPassSlots + sizeof(int) * kMaxPassSlots;
    }
};

template <typename T, int K, int R>
__global__ void __launch_bounds__(1 << (K - R))
    k_fused_rev(const amp_t<T> *__restrict__ phi_src, amp_t<T> *__restrict__ phi_dst,
                amp_t<T> *__restrict__ lam, const FPass *__restrict__ passes, int pi,
                const FStage *__restrict__ stages, const FOp *__restrict__ ops,
                const int *__restrict__ slot_map, const T *__restrict__ mats, uint64_t n_tiles,
                double *__restrict__ partials, int nb) {
    using A = amp_t<T>;
    using IO = TileIO<T, K>;
    constexpr int AB = FT<T>::AB, NT = 1 << (K - R), NA = 1 << R, NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    A *tphi = reinterpret_cast<A *>(smem);
    A *tlam = tphi + (1 << K);
    uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + 2 * (size_t)(1 << K) * AB);
    FStage *sst = reinterpret_cast<FStage *>(row_off + IO::ROWS);
    FOp *sop = reinterpret_cast<FOp *>(sst + kMaxPassStages);
    double *acc = reinterpret_cast<double *>(sop + kMaxPassOps);
    int *smap = reinterpret_cast<int *>(acc + NW * kMaxPassSlots);
    const FPass &P = passes[pi];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_stage = P.n_rstage, n_ls = P.n_lslots;
    load_pass<T, K>(P, P.rstage0, n_stage, stages, ops, sst, sop, row_off, tid, NT);
    for (int i = tid; i < NW * n_ls; i += NT) acc[i] = 0.0;
    for (int i = tid; i < n_ls; i += NT) smap[i] = slot_map[P.slotmap0 + i];
    const int op_base = n_stage ? stages[P.rstage0].op0 : 0;
    const int n_nontile = P.n_nontile;
    __syncthreads();
    for (uint64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const uint64_t base = tile_base(ti, P.nontile, n_nontile);
        IO::load(tphi, phi_src, base, row_off, tid, NT);
        IO::load(tlam, lam, base, row_off, tid, NT);
        __syncthreads();
        for (int s = 0; s < n_stage; ++s) {
            const FStage &st = sst[s];
            uint32_t sb = 0;
            uint64_t gb = base;
#pragma unroll
            for (int b = 0; b < K - R; ++b)
                if ((tid >> b) & 1) sb ^= st.thr_sw[b], gb |= st.thr_g[b];
            uint32_t w[R];
#pragma unroll
            for (int k = 0; k < R; ++k) w[k] = st.reg_sw[k];
            A a[NA], l[NA];
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                uint32_t ad = sb;
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if ((j >> k) & 1) ad ^= w[k];
                a[j] = tphi[ad];
                l[j] = tlam[ad];
            }
            const int o_end = st.op0 - op_base + st.n_op;
            for (int o = st.op0 - op_base; o < o_end; ++o) {
                const FOp &op = sop[o];
                const T *m = mats + 8 * (size_t)op.gate;
                T v1 = 0;
                bool red1 = false;
                switch (op.type) {
                case OP_RY: {
                    const T c = m[0], s_ = m[4];
                    with_k<R>(op.k, [&](auto kb) { v1 = rev_ry<decltype(kb)::value, NA, T>(a, l, c, s_); });
                    red1 = true;
                    break;
                }
                case OP_RX: {
                    const Mat2<T> ud = dagger<T>(mat_of<T>(m));
                    with_k<R>(op.k, [&](auto kb) { v1 = rev_rx<decltype(kb)::value, NA, T>(a, l, ud); });
                    red1 = true;
                    break;
                }
                case OP_U3: {
                    const Mat2<T> ud = dagger<T>(mat_of<T>(m));
                    T v8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    with_k<R>(op.k, [&](auto kb) { rev_u3<decltype(kb)::value, NA, T>(a, l, ud, v8); });
                    const T tot = warp_reduce8<T>(v8);
                    if ((lane & 3) == 0) {
                        const int vi = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                        acc[warp * n_ls + op.lslot + vi] += (double)tot;
                    }
                    break;
                }
                case OP_RZ_REG: {
                    const amp_t<T> q0 = mk<T>(m[0], -m[1]), q1 = mk<T>(m[6], -m[7]);
                    with_k<R>(op.k, [&](auto kb) { v1 = rev_rzr<decltype(kb)::value, NA, T>(a, l, q0, q1); });
                    red1 = true;
                    break;
                }
                case OP_RZ_THR: {
                    const bool b = (gb & op.g0) != 0;
                    const amp_t<T> q = b ? mk<T>(m[6], -m[7]) : mk<T>(m[0], -m[1]);
                    v1 = rev_rzt<NA, T>(a, l, q, b);
                    red1 = true;
                    break;
                }
                case OP_CZ: {
                    const bool ok = (op.rm0 || (gb & op.g0)) && (op.rm1 || (gb & op.g1));
                    op_cz<NA, T>(a, op.rm0 | op.rm1, ok);
                    op_cz<NA, T>(l, op.rm0 | op.rm1, ok);
                    break;
                }
                case OP_CNOT: {
                    const bool c = (gb & op.g0) != 0;
                    with_k<R>(op.k, [&](auto kb) {
                        op_cnot<decltype(kb)::value, NA, T>(a, op.rm0, c);
                        op_cnot<decltype(kb)::value, NA, T>(l, op.rm0, c);
                    });
                    break;
                }
                default:
                    break;
                }
                if (red1) {
                    const T tot = warp_tree<T>(v1);
                    if (lane == 0) acc[warp * n_ls + op.lslot] += (double)tot;
                }
            }
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                uint32_t ad = sb;
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if ((j >> k) & 1) ad ^= w[k];
                tphi[ad] = a[j];
                tlam[ad] = l[j];
            }
            __syncthreads();
        }
        IO::store(tphi, phi_dst, base, row_off, tid, NT);
        IO::store(tlam, lam, base, row_off, tid, NT);
        __syncthreads();
    }
    __syncthreads();
    for (int i = tid; i < n_ls; i += NT) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += acc[w * n_ls + i];
        partials[(size_t)smap[i] * nb + blockIdx.x] = s;
    }
}

// ------------------------------------------------------------------ Hamiltonian pass
template <typename T, int K>
struct HamCfg {
    static constexpr int NT = 256;
    static constexpr size_t smem() {
        return (size_t)(1 << K) * FT<T>::AB + sizeof(uint64_t) * (1 << (K - FT<T>::L));
    }
};

template <typename T, int K>
__global__ void __launch_bounds__(256)
    k_fused_ham(const amp_t<T> *__restrict__ psi, amp_t<T> *__restrict__ lam,
                const HPass *__restrict__ hp, int pi, const HGroup *__restrict__ groups,
                const HTerm *__restrict__ terms, uint64_t n_tiles, double *__restrict__ partials, int nb) {
    using A = amp_t<T>;
    using IO = TileIO<T, K>;
    constexpr int AB = FT<T>::AB, L = FT<T>::L, NT = 256;
    extern __shared__ __align__(16) unsigned char smem[];
    A *tile = reinterpret_cast<A *>(smem);
    uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + (size_t)(1 << K) * AB);
    __shared__ double wsum[NT / 32];
    const HPass &P = hp[pi];
    const int tid = threadIdx.x;
    for (int r = tid; r < IO::ROWS; r += NT) {
        uint64_t off = 0;
        for (int i = 0; i < K - L; ++i)
            if ((r >> i) & 1) off |= 1ull << P.high[i];
        row_off[r] = off;
    }
    const int g0 = P.group0, ng = P.n_group;
    const bool first = P.first;
    double eacc = 0.0;
    __syncthreads();
    for (uint64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const uint64_t base = tile_base(ti, P.nontile, P.n_nontile);
        IO::load(tile, psi, base, row_off, tid, NT);
        __syncthreads();
        T run = 0;
        for (int c = tid; c < IO::CHUNKS; c += NT) {
            const int row = c / IO::CPR, col = c % IO::CPR;
            const uint32_t t0 = (uint32_t)(row << L) | (uint32_t)(col * IO::CA);
            const uint64_t gidx0 = base | row_off[row] | (uint64_t)(col * IO::CA);
            union {
                float4 f;
                A a[IO::CA];
            } out;
            A mine[IO::CA];
            if (!first) out.f = __ldcs(reinterpret_cast<const float4 *>(lam + gidx0));
#pragma unroll
            for (int e = 0; e < IO::CA; ++e) {
                mine[e] = tile[swz<AB>(t0 + e)];
                if (first) out.a[e] = mk<T>((T)0, (T)0);
            }
            for (int g = g0; g < g0 + ng; ++g) {
                const HGroup G = groups[g];
#pragma unroll
                for (int e = 0; e < IO::CA; ++e) {
                    const uint64_t gi = gidx0 + e;
                    const A src = tile[swz<AB>((t0 + e) ^ G.xl)];
                    T fr = 0, fi = 0;
                    for (int k = G.term0; k < G.term0 + G.n_term; ++k) {
                        const HTerm tm = terms[k];
                        const bool odd = __popcll(gi & tm.z) & 1;
                        T wr, wi;
                        if constexpr (sizeof(T) == 4) wr = tm.fr, wi = tm.fi;
                        else wr = tm.wr, wi = tm.wi;
                        fr += odd ? -wr : wr;
                        fi += odd ? -wi : wi;
                    }
                    const A d = cmul<T>(mk<T>(fr, fi), src);
                    out.a[e] = cadd<T>(out.a[e], d);
                    run += mine[e].x * d.x + mine[e].y * d.y;
                }
            }
            __stcs(reinterpret_cast<float4 *>(lam + gidx0), out.f);
        }
        eacc += (double)warp_tree<T>(run);  // lane 0's copy is used below
        __syncthreads();
    }
    if ((tid & 31) == 0) wsum[tid >> 5] = eacc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += wsum[w];
        partials[(size_t)P.eslot * nb + blockIdx.x] = s;
    }
}

// ------------------------------------------------------------------ launchers
template <typename Kern>
static void set_smem(Kern k, size_t bytes) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int K, int R>
static void fwd_t(const void *src, void *dst, const FPass *passes, int pi, const FStage *st,
                  const FOp *ops, const void *mats, uint64_t n_tiles, int grid, cudaStream_t s) {
    constexpr size_t sm = FwdCfg<T, K, R>::smem();
    static bool once = false;
    if (!once) set_smem(k_fused_fwd<T, K, R>, sm), once = true;
    k_fused_fwd<T, K, R><<<grid, FwdCfg<T, K, R>::NT, sm, s>>>(
        (const amp_t<T> *)src, (amp_t<T> *)dst, passes, pi, st, ops, (const T *)mats, n_tiles);
}

template <typename T, int K, int R>
static void rev_t(const void *phi_src, void *phi_dst, void *lam, const FPass *passes, int pi,
                  const FStage *st, const FOp *ops, const int *slot_map, const void *mats,
                  uint64_t n_tiles, double *partials, int nb, cudaStream_t s) {
    constexpr size_t sm = RevCfg<T, K, R>::smem();
    static bool once = false;
    if (!once) set_smem(k_fused_rev<T, K, R>, sm), once = true;
    k_fused_rev<T, K, R><<<nb, RevCfg<T, K, R>::NT, sm, s>>>(
        (const amp_t<T> *)phi_src, (amp_t<T> *)phi_dst, (amp_t<T> *)lam, passes, pi, st, ops,
        slot_map, (const T *)mats, n_tiles, partials, nb);
}

template <typename T, int K>
static void ham_t(const void *psi, void *lam, const HPass *hp, int pi, const HGroup *groups,
                  const HTerm *terms, uint64_t n_tiles, double *partials, int nb, cudaStream_t s) {
    constexpr size_t sm = HamCfg<T, K>::smem();
    static bool once = false;
    if (!once) set_smem(k_fused_ham<T, K>, sm), once = true;
    k_fused_ham<T, K><<<nb, 256, sm, s>>>((const amp_t<T> *)psi, (amp_t<T> *)lam, hp, pi, groups,
                                           terms, n_tiles, partials, nb);
}

// Supported tile sizes: complex64 K = 10..13 (R_fwd = 5, R_rev = 4);
// complex128 K = 10..12 (R_fwd = 4, R_rev = 3).
void launch_fused_fwd(bool dbl, int K, const void *src, void *dst, const FPass *passes, int pi,
                      const FStage *st, const FOp *ops, const void *mats, uint64_t n_tiles, int grid,
                      cudaStream_t s) {
    if (!dbl) {
        switch (K) {
        case 10: fwd_t<float, 10, 5>(src, dst, passes, pi, st, ops, mats, n_tiles, grid, s); break;
        case 11: fwd_t<float, 11, 5>(src, dst, passes, pi, st, ops, mats, n_tiles, grid, s); break;
        case 12: fwd_t<float, 12, 5>(src, dst, passes, pi, st, ops, mats, n_tiles, grid, s); break;
        case 13: fwd_t<float, 13, 5>(src, dst, passes, pi, st, ops, mats, n_tiles, grid, s); break;
        default: break;
        }
    } else {
        switch (K) {
        case 10: fwd_t<double, 10, 4>(src, dst, passes, pi, st, ops, mats, n_tiles, grid, s); break;
        case 11: fwd_t<double, 11, 4>(src, dst, passes, pi, st, ops, mats, n_tiles, grid, s); break;
        case 12: fwd_t<double, 12, 4>(src, dst, passes, pi, st, ops, mats, n_tiles, grid, s); break;
        default: break;
        }
    }
}

void launch_fused_rev(bool dbl, int K, const void *phi_src, void *phi_dst, void *lam,
                      const FPass *passes, int pi, const FStage *st, const FOp *ops,
                      const int *slot_map, const void *mats, uint64_t n_tiles, double *partials,
                      int nb, cudaStream_t s) {
#define VQG_REV(TT, KK, RR) \
    rev_t<TT, KK, RR>(phi_src, phi_dst, lam, passes, pi, st, ops, slot_map, mats, n_tiles, partials, nb, s)
    if (!dbl) {
        switch (K) {
        case 10: VQG_REV(float, 10, 4); break;
        case 11: VQG_REV(float, 11, 4); break;
        case 12: VQG_REV(float, 12, 4); break;
        case 13: VQG_REV(float, 13, 4); break;
        default: break;
        }
    } else {
        switch (K) {
        case 10: VQG_REV(double, 10, 3); break;
        case 11: VQG_REV(double, 11, 3); break;
        case 12: VQG_REV(double, 12, 3); break;
        default: break;
        }
    }
#undef VQG_REV
}

void launch_fused_ham(bool dbl, int K, const void *psi, void *lam, const HPass *hp, int pi,
                      const HGroup *groups, const HTerm *terms, uint64_t n_tiles, double *partials,
                      int nb, cudaStream_t s) {
    if (!dbl) {
        switch (K) {
        case 10: ham_t<float, 10>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 11: ham_t<float, 11>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 12: ham_t<float, 12>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 13: ham_t<float, 13>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        default: break;
        }
    } else {
        switch (K) {
        case 10: ham_t<double, 10>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 11: ham_t<double, 11>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 12: ham_t<double, 12>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        default: break;
        }
    }
}

}  // namespace vqg
