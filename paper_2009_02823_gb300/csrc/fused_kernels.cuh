// Tile-fused sweeps (the gate-fusion scheme of the GB300 design; the paper's
// algorithm only needs "apply gate" primitives, Sec. 2.1, and leaves their fusion to
// the simulator).
//
//   k_fused_fwd : one forward pass -- every tile of 2^K amplitudes is read from HBM once,
//                 a run of gates is applied in shared memory / registers, and the tile
//                 is written once (Algorithm 1's forward sweep, many gates per state traversal).
//   k_fused_rev : one reverse pass -- phi and lambda tiles are read once, and for each
//                 gate of the run in reverse order the kernel reduces the gradient sums
//                 from (phi_{i+1}, lambda_i) and un-applies U_i^dagger to both
//                 (Algorithm 1's reverse loop, with App. A's dR = -(i/2) sigma R so that
//                 mu = dU phi is never formed; App. B.1 for U3).
//   k_fused_ham : one Hamiltonian pass -- the Pauli groups whose flip mask lies inside
//                 the tile, lambda (+)= sum_g f_g(j^x) psi[j^x], with E = Re<psi|lambda>.
//
// Reduction precision (complex64 amplitudes): products in FP32, per-thread runs of at
// most 16 terms in FP32; in the reverse pass the block's per-thread partials of one tile
// are summed in FP32 (lane runs of NT/32 values, then the 32-lane tree) and added to an
// FP64 accumulator per tile; block and grid levels are FP64.
//
// complex64 arithmetic uses packed FP32 pairs (sm_100 and later) where one instruction can
// update the real and imaginary parts together: RY ops in a scaled form with one packed
// multiply-add per output (the stage carries the dropped factor, see load_prog), and the
// reverse pass's diagonal multiplies whose factor is shared by phi and lambda.  complex128
// tiles compute in FP64 or, by option, in float-float (df.cuh).
#pragma once
#include <type_traits>

#include "df.cuh"
#include "fused.h"
#include "kernels.h"

namespace vqg {

// Per arithmetic type: row qubits L (one 128-byte row), bytes per amplitude in shared
// memory, the gate-table element type, and whether global amplitudes are converted on
// the way in and out (float-float tiles of complex128 states).
template <typename T> struct FT;
template <> struct FT<float> { static constexpr int L = 4, AB = 8; using mat_t = float; static constexpr bool conv = false; };
template <> struct FT<double> { static constexpr int L = 3, AB = 16; using mat_t = double; static constexpr bool conv = false; };
template <> struct FT<df> { static constexpr int L = 3, AB = 16; using mat_t = double; static constexpr bool conv = true; };

template <typename T> VQG_DEV T shfl(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <> VQG_DEV df shfl<df>(df v, int m) {
    return df(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

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

// a * b + c in the tile arithmetic
template <typename T> VQG_DEV T fma_t(T a, T b, T c);
template <> VQG_DEV float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <> VQG_DEV double fma_t<double>(double a, double b, double c) { return ::fma(a, b, c); }
template <> VQG_DEV df fma_t<df>(df a, df b, df c) { return vqg::fma(a, b, c); }

// v with its sign flipped where s (0 or 0x80000000) is set: a logic op on the sign bit.
template <typename T> VQG_DEV T flip_sign(T v, uint32_t s);
template <> VQG_DEV float flip_sign<float>(float v, uint32_t s) { return __uint_as_float(__float_as_uint(v) ^ s); }
template <> VQG_DEV double flip_sign<double>(double v, uint32_t s) {
    return __hiloint2double(__double2hiint(v) ^ (int)s, __double2loint(v));
}
template <> VQG_DEV df flip_sign<df>(df v, uint32_t s) { return df(flip_sign<float>(v.hi, s), flip_sign<float>(v.lo, s)); }

// ------------------------------------------------------------------ gate ops (forward)
template <int KB, int NA, typename T>
VQG_DEV void op_ry(amp_t<T> (&a)[NA], T c, T s) {
    if constexpr (std::is_same<T, float>::value) {  // real factors: packed FP32 pairs
        const float2 cc = make_float2(c, c), ss = make_float2(s, s), ns = make_float2(-s, -s);
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if (j & (1 << KB)) continue;
            const int j1 = j | (1 << KB);
            const float2 x = a[j], y = a[j1];
            a[j] = __ffma2_rn(cc, x, __fmul2_rn(ns, y));
            a[j1] = __ffma2_rn(ss, x, __fmul2_rn(cc, y));
        }
    } else if constexpr (std::is_same<T, df>::value) {  // packed float-float (re, im) lanes
        const float2 ch = make_float2(c.hi, c.hi), cl = make_float2(c.lo, c.lo);
        const float2 sh = make_float2(s.hi, s.hi), sl = make_float2(s.lo, s.lo);
        const float2 nsh = make_float2(-s.hi, -s.hi), nsl = make_float2(-s.lo, -s.lo);
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if (j & (1 << KB)) continue;
            const int j1 = j | (1 << KB);
            const dfp x = to_dfp(a[j]), y = to_dfp(a[j1]);
            a[j] = from_dfp(fma2(ch, cl, x, mul2(nsh, nsl, y)));
            a[j1] = from_dfp(fma2(sh, sl, x, mul2(ch, cl, y)));
        }
    } else {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if (j & (1 << KB)) continue;
            const int j1 = j | (1 << KB);
            const amp_t<T> x = a[j], y = a[j1];
            a[j] = mk<T>(c * x.x - s * y.x, c * x.y - s * y.y);
            a[j1] = mk<T>(s * x.x + c * y.x, s * x.y + c * y.y);
        }
    }
}

// Range of the scaled form: each scaled RY drops a factor k with |k| >= 2^-1/2, so a stage
// of m RY ops holds amplitudes up to 2^(m/2) times their true values (at most 1 in
// magnitude for a normalised state) and the reverse pass scales its reduction partials by
// K^2 >= 2^-m.  A forward stage holds at most kMaxPassOps ops and a reverse stage at most
// kMaxStageValues RY ops (one reduction value each); both bounds keep the held values and
// K^2 inside FP32's normal range (2^-126 .. 2^128) with a wide margin.
static_assert(kMaxPassOps / 2 <= 100, "forward scaled-RY stages could leave FP32's range");
static_assert(kMaxStageValues <= 100, "reverse scaled-RY stages could leave FP32's range");

// Whether a stage's amplitudes carry a scale to undo at the scatter (complex64 only).
template <typename T> VQG_DEV bool scaled_stage(T kacc) {
    if constexpr (std::is_same<T, float>::value) return kacc != 1.f;
    else return false;
}

// complex64 RY without its scale factor k (see load_prog): each output is one packed
// multiply-add and equals the true output divided by k; the caller multiplies the stage's
// amplitudes by the product of the k at the scatter.  C-form: (a0 - r a1, a1 + r a0);
// S-form: (r a0 - a1, a0 + r a1).
template <int KB, int NA>
VQG_DEV void op_ry_scaled(float2 (&a)[NA], float r, bool sform) {
    const float2 rr = make_float2(r, r), nr = make_float2(-r, -r);
    if (!sform) {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if (j & (1 << KB)) continue;
            const int j1 = j | (1 << KB);
            const float2 x = a[j], y = a[j1];
            a[j] = __ffma2_rn(nr, y, x);
            a[j1] = __ffma2_rn(rr, x, y);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if (j & (1 << KB)) continue;
            const int j1 = j | (1 << KB);
            const float2 x = a[j], y = a[j1];
            a[j] = __ffma2_rn(rr, x, make_float2(-y.x, -y.y));
            a[j1] = __ffma2_rn(rr, y, x);
        }
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

// Controlled 2x2 (controlled rotations, phase gates): u on the pair where the control
// is set -- register mask rc, else the thread-level flag thr_c.
template <int KB, int NA, typename T>
VQG_DEV void op_cgen(amp_t<T> (&a)[NA], const Mat2<T> &u, uint32_t rc, bool thr_c) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        const bool c = rc ? ((j & rc) != 0) : thr_c;
        if (c) apply2<T>(u, a[j], a[j | (1 << KB)]);
    }
}

// Control flag of an op whose control is not a register bit (cq < 0: no control).
VQG_DEV bool thread_control(const FOp &op, uint64_t gb) {
    return op.rm0 ? false : (op.cq < 0 ? true : ((gb >> op.cq) & 1ull) != 0);
}

template <typename T> VQG_DEV Mat2<T> mat_of(const amp_t<T> *__restrict__ m) {
    Mat2<T> u;
#pragma unroll
    for (int k = 0; k < 4; ++k) u.m[k] = m[k];
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

// Sign pattern over register indices j < 2^R: bit j = parity(j & c).
VQG_DEV uint32_t walsh_bits(uint32_t c) {
    uint32_t w = 0;
    if (c & 1u) w ^= 0xAAAAAAAAu;
    if (c & 2u) w ^= 0xCCCCCCCCu;
    if (c & 4u) w ^= 0xF0F0F0F0u;
    if (c & 8u) w ^= 0xFF00FF00u;
    if (c & 16u) w ^= 0xFFFF0000u;
    return w;
}

// ------------------------------------------------------------------ pass program in smem
// One pass's register-stage program (forward or reverse), staged in shared memory by
// every block at launch: stages, ops, diagonal blocks and their items, the gate
// matrices of the ops (U; the reverse kernel takes U^dagger of them), the RZ phases of
// the items (conjugated for the reverse), and each diagonal block's 2^R-entry table
// (RZ phases on register bits times CZ signs between register bits).
// Byte offsets of a pass program's tables in shared memory for the counts it is sized
// for; host code sizes the specialised kernels' shared memory with the same function.
struct ProgOffsets {
    size_t st, op, dg, it, prm, iph, tab, ti, bytes;
};
__host__ __device__ constexpr size_t prog_align(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ constexpr ProgOffsets prog_offsets(size_t ab, int R, int stages, int ops, int diags, int items) {
    ProgOffsets o{};
    o.st = 0;
    o.op = prog_align(o.st + sizeof(FStage) * stages);
    o.dg = prog_align(o.op + sizeof(FOp) * ops);
    o.it = prog_align(o.dg + sizeof(FDiag) * diags);
    o.prm = prog_align(o.it + sizeof(FDItem) * items);
    o.iph = prog_align(o.prm + ab * 4 * ops);
    o.tab = prog_align(o.iph + ab * 2 * items);
    o.ti = prog_align(o.tab + ab * ((size_t)1 << R) * diags);
    o.bytes = prog_align(o.ti + sizeof(uint32_t) * items);
    return o;
}

template <typename T, int R>
struct Prog {
    static constexpr int AB = FT<T>::AB;
    // shared-memory layout for the program budget C
    template <typename C = FullCaps>
    struct Layout {
        static constexpr ProgOffsets po = prog_offsets(AB, R, C::stages, C::ops, C::diags, C::items);
        static constexpr size_t o_st = po.st, o_op = po.op, o_dg = po.dg, o_it = po.it, o_prm = po.prm,
                                o_iph = po.iph, o_tab = po.tab, o_ti = po.ti, bytes = po.bytes;
    };

    FStage *st;
    FOp *op;
    FDiag *dg;
    FDItem *it;
    amp_t<T> *prm, *iph, *tab;
    uint32_t *ti;  // per item, packed for the per-thread factor: type | q0 << 8 | q1 << 16 | k0 << 24
    int op_base, item_base;

    template <typename C = FullCaps>
    VQG_DEV void bind(unsigned char *p) {
        using Lo = Layout<C>;
        st = reinterpret_cast<FStage *>(p + Lo::o_st);
        op = reinterpret_cast<FOp *>(p + Lo::o_op);
        dg = reinterpret_cast<FDiag *>(p + Lo::o_dg);
        it = reinterpret_cast<FDItem *>(p + Lo::o_it);
        prm = reinterpret_cast<amp_t<T> *>(p + Lo::o_prm);
        iph = reinterpret_cast<amp_t<T> *>(p + Lo::o_iph);
        tab = reinterpret_cast<amp_t<T> *>(p + Lo::o_tab);
        ti = reinterpret_cast<uint32_t *>(p + Lo::o_ti);
    }
};

template <typename W>
VQG_DEV void copy_words(W *dst, const W *__restrict__ src, int count, int tid, int nt) {
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    const int words = count * (int)(sizeof(W) / 4);
    for (int i = tid; i < words; i += nt) d[i] = s[i];
}

template <typename T, int R>
VQG_DEV void load_prog(Prog<T, R> &pg, int s0, int ns, int d0, int nd, const FStage *__restrict__ stages,
                       const FOp *__restrict__ ops, const FDiag *__restrict__ diags,
                       const FDItem *__restrict__ items, const typename FT<T>::mat_t *__restrict__ mats, bool reverse,
                       int tid, int nt) {
    const int op0 = ns ? stages[s0].op0 : 0;
    const int n_op = ns ? stages[s0 + ns - 1].op0 + stages[s0 + ns - 1].n_op - op0 : 0;
    const int it0 = nd ? diags[d0].item0 : 0;
    const int n_it = nd ? diags[d0 + nd - 1].item0 + diags[d0 + nd - 1].n_item - it0 : 0;
    pg.op_base = op0;
    pg.item_base = it0;
    copy_words(pg.st, stages + s0, ns, tid, nt);
    copy_words(pg.op, ops + op0, n_op, tid, nt);
    copy_words(pg.dg, diags + d0, nd, tid, nt);
    copy_words(pg.it, items + it0, n_it, tid, nt);
    for (int o = tid; o < n_op; o += nt) {
        const FOp op = ops[op0 + o];
        const int g = op.gate;
        if (g < 0) continue;
        const typename FT<T>::mat_t *m = mats + 8 * (size_t)g;
        if (op.type == OP_RY) {  // (cos, sin) of the real rotation in one slot
            pg.prm[4 * o] = mk<T>((T)m[0], (T)m[4]);
            if constexpr (std::is_same<T, float>::value) {
                // scaled form: RY = k [[1, -r], [r, 1]] (k = c, r = s / c) when |c| >= |s|,
                // else k [[r, -1], [1, r]] (k = s, r = c / s); |r| <= 1.  Slot 1: (r, form),
                // slot 2: (k, k^2), computed in FP64 from the table entries, rounded once.
                const double c = m[0], sn = m[4];
                const bool sform = std::fabs(sn) > std::fabs(c);
                const double k = sform ? sn : c, r = sform ? c / sn : sn / c;
                pg.prm[4 * o + 1] = mk<T>((T)r, sform ? (T)1 : (T)0);
                pg.prm[4 * o + 2] = mk<T>((T)k, (T)(k * k));
            }
            continue;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) pg.prm[4 * o + e] = mk<T>((T)m[2 * e], (T)m[2 * e + 1]);
    }
    for (int i = tid; i < n_it; i += nt) {
        const FDItem x = items[it0 + i];
        // qubit of a single-bit mask (thread-level qubits of RZ_THR / CZ_RT / CZ_TT)
        const uint32_t q0 = x.g0 ? (uint32_t)__ffsll((long long)x.g0) - 1u : 0u;
        const uint32_t q1 = x.g1 ? (uint32_t)__ffsll((long long)x.g1) - 1u : 0u;
        pg.ti[i] = (uint32_t)x.type | (q0 << 8) | (q1 << 16) | ((uint32_t)(x.k0 & 0xff) << 24);
        if (x.type != DI_RZ_REG && x.type != DI_RZ_THR) continue;
        const typename FT<T>::mat_t *m = mats + 8 * (size_t)x.gate;
        const T sg = reverse ? (T)-1 : (T)1;
        pg.iph[2 * i] = mk<T>((T)m[0], sg * (T)m[1]);
        pg.iph[2 * i + 1] = mk<T>((T)m[6], sg * (T)m[7]);
    }
    __syncthreads();
    constexpr int NA = 1 << R;
    for (int e = tid; e < nd * NA; e += nt) {
        const int d = e / NA, j = e % NA;
        const FDiag D = pg.dg[d];
        amp_t<T> v = mk<T>((T)1, (T)0);
        for (int i = D.item0 - it0; i < D.item0 - it0 + D.n_item; ++i) {
            const FDItem &x = pg.it[i];
            if (x.type == DI_RZ_REG) v = cmul<T>(((j >> x.k0) & 1) ? pg.iph[2 * i + 1] : pg.iph[2 * i], v);
            else if (x.type == DI_CZ_RR && ((j >> x.k0) & 1) && ((j >> x.k1) & 1)) v = neg<T>(v);
        }
        pg.tab[e] = v;
    }
}

// Per-thread factor of a diagonal block: tau (phases of RZ on thread-level qubits and
// CZ signs between thread-level qubits) and the register mask whose parity flips sign
// (CZ between a register bit and a set thread-level bit).
template <typename T, int R>
VQG_DEV void diag_thread(const Prog<T, R> &pg, const FDiag &D, uint64_t gb, amp_t<T> &tau, uint32_t &c) {
    tau = mk<T>((T)1, (T)0);
    c = 0;
    const int i0 = D.item0 - pg.item_base + D.thr0;  // thread-level items only
    for (int i = i0; i < i0 + D.n_thr; ++i) {
        const uint32_t p = pg.ti[i];
        const uint32_t type = p & 0xffu, b0 = (uint32_t)(gb >> ((p >> 8) & 0xffu)) & 1u;
        if (type == DI_RZ_THR) {
            tau = cmul<T>(b0 ? pg.iph[2 * i + 1] : pg.iph[2 * i], tau);
        } else if (type == DI_CZ_TT) {
            if (b0 & (uint32_t)(gb >> ((p >> 16) & 0xffu))) tau = neg<T>(tau);
        } else {  // DI_CZ_RT
            if (b0) c ^= 1u << (p >> 24);
        }
    }
}

// Multiply by the block's table with the per-thread sign pattern; the per-thread
// phase tau is not applied here but folded into the stage's pending phase: a common
// factor on all of a thread's amplitudes commutes with every later op of the stage
// (they act within the thread's amplitudes) and is applied once before the scatter.
template <int NA, typename T>
VQG_DEV void diag_apply(amp_t<T> (&a)[NA], const amp_t<T> *__restrict__ tab, uint32_t c, bool has_rt) {
    if (has_rt) {  // block-uniform: sign pattern only where a register-thread CZ exists
        const uint32_t w = walsh_bits(c);
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            amp_t<T> d = tab[j];
            if ((w >> j) & 1u) d = neg<T>(d);
            a[j] = cmul<T>(d, a[j]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NA; ++j) a[j] = cmul<T>(tab[j], a[j]);
    }
}

template <int R, int NA, typename T>
VQG_DEV void apply_fwd_op(amp_t<T> (&a)[NA], const Prog<T, R> &pg, int o, uint64_t gb, amp_t<T> &phase,
                          T &kacc) {
    const FOp op = pg.op[o];
    const amp_t<T> *m = pg.prm + 4 * o;
    switch (op.type) {
    case OP_RY: {
        if constexpr (std::is_same<T, float>::value) {  // scaled form; k joins the stage's factor
            const float2 p1 = m[1];
            with_k<R>(op.k, [&](auto kb) { op_ry_scaled<decltype(kb)::value, NA>(a, p1.x, p1.y != 0.f); });
            kacc *= m[2].x;
        } else {
            const amp_t<T> cs = m[0];
            with_k<R>(op.k, [&](auto kb) { op_ry<decltype(kb)::value, NA, T>(a, cs.x, cs.y); });
        }
        break;
    }
    case OP_RX:
    case OP_U3: {
        const Mat2<T> u = mat_of<T>(m);
        with_k<R>(op.k, [&](auto kb) { op_gen<decltype(kb)::value, NA, T>(a, u); });
        break;
    }
    case OP_CNOT: {
        const bool c = op.rm0 ? false : ((gb >> op.cq) & 1ull) != 0;
        with_k<R>(op.k, [&](auto kb) { op_cnot<decltype(kb)::value, NA, T>(a, op.rm0, c); });
        break;
    }
    case OP_CRX:
    case OP_CRY:
    case OP_CRZ:
    case OP_PH: {
        const Mat2<T> u = mat_of<T>(m);
        const bool c = thread_control(op, gb);
        with_k<R>(op.k, [&](auto kb) { op_cgen<decltype(kb)::value, NA, T>(a, u, op.rm0, c); });
        break;
    }
    case OP_DIAG: {
        amp_t<T> tau;
        uint32_t c;
        diag_thread<T, R>(pg, pg.dg[op.diag], gb, tau, c);
        phase = cmul<T>(tau, phase);
        diag_apply<NA, T>(a, pg.tab + op.diag * NA, c, pg.dg[op.diag].has_rt != 0);
        break;
    }
    default:
        break;
    }
}

// ------------------------------------------------------------------ gate ops (reverse)
// Balanced pairwise sum (short dependency chains; N a power of two).  Consumes x.
template <int N, typename T>
VQG_DEV T tree_sum(T (&x)[N], int n = N) {  // the first n entries (n a power of two, <= N)
#pragma unroll
    for (int s = 1; s < N; s *= 2)
#pragma unroll
        for (int i = 0; i + s < N; i += 2 * s)
            if (i + s < n) x[i] += x[i + s];
    return x[0];
}

// complex64 RY^dagger without its scale factor k, on phi and lambda: C-form
// (a0 + r a1, a1 - r a0), S-form (r a0 + a1, r a1 - a0).  Returns the raw partial of
// Im <lambda|Y|phi> from the inputs, which hold the true values divided by the stage's
// product K of the k so far (the caller multiplies the partial by K^2).
template <int KB, int NA, bool SFORM>
VQG_DEV float rev_ry_scaled_form(float2 (&a)[NA], float2 (&l)[NA], float r) {
    const float2 rr = make_float2(r, r), nr = make_float2(-r, -r);
    float2 P[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, Q[2] = {P[0], P[1]};
    int q = 0;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        const int j1 = j | (1 << KB);
        const float2 a0 = a[j], a1 = a[j1], l0 = l[j], l1 = l[j1];
        P[q & 1] = __ffma2_rn(l1, a0, P[q & 1]);
        Q[q & 1] = __ffma2_rn(l0, a1, Q[q & 1]);
        ++q;
        if constexpr (!SFORM) {
            a[j] = __ffma2_rn(rr, a1, a0);
            a[j1] = __ffma2_rn(nr, a0, a1);
            l[j] = __ffma2_rn(rr, l1, l0);
            l[j1] = __ffma2_rn(nr, l0, l1);
        } else {
            a[j] = __ffma2_rn(rr, a0, a1);
            a[j1] = __ffma2_rn(rr, a1, make_float2(-a0.x, -a0.y));
            l[j] = __ffma2_rn(rr, l0, l1);
            l[j1] = __ffma2_rn(rr, l1, make_float2(-l0.x, -l0.y));
        }
    }
    const float2 p = __fadd2_rn(P[0], P[1]), t = __fadd2_rn(Q[0], Q[1]);
    return (p.x + p.y) - (t.x + t.y);
}
template <int KB, int NA>
VQG_DEV float rev_ry_scaled(float2 (&a)[NA], float2 (&l)[NA], float r, bool sform) {
    return sform ? rev_ry_scaled_form<KB, NA, true>(a, l, r) : rev_ry_scaled_form<KB, NA, false>(a, l, r);
}

// Each returns the thread's partial of the gate's reduction value(s) computed from
// (phi_{i+1} = a, lambda_i = l) before un-applying U^dagger to both.
template <int KB, int NA, typename T>
VQG_DEV T rev_ry(amp_t<T> (&a)[NA], amp_t<T> (&l)[NA], T c, T s) {
    if constexpr (std::is_same<T, float>::value) {
        // Packed FP32 pairs: the RY^dagger updates have real factors, and the reduction
        // keeps sum(l1 * a0) and sum(l0 * a1) component-wise (two chains each), combined
        // as (P.x + P.y) - (Q.x + Q.y) at the end.
        const float2 cc = make_float2(c, c), ss = make_float2(s, s), ns = make_float2(-s, -s);
        float2 P[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, Q[2] = {P[0], P[1]};
        int q = 0;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if (j & (1 << KB)) continue;
            const int j1 = j | (1 << KB);
            const float2 a0 = a[j], a1 = a[j1], l0 = l[j], l1 = l[j1];
            P[q & 1] = __ffma2_rn(l1, a0, P[q & 1]);
            Q[q & 1] = __ffma2_rn(l0, a1, Q[q & 1]);
            ++q;
            a[j] = __ffma2_rn(cc, a0, __fmul2_rn(ss, a1));
            a[j1] = __ffma2_rn(cc, a1, __fmul2_rn(ns, a0));
            l[j] = __ffma2_rn(cc, l0, __fmul2_rn(ss, l1));
            l[j1] = __ffma2_rn(cc, l1, __fmul2_rn(ns, l0));
        }
        const float2 p = __fadd2_rn(P[0], P[1]), r = __fadd2_rn(Q[0], Q[1]);
        return (p.x + p.y) - (r.x + r.y);
    } else {
        T pv[NA / 2];
        int q = 0;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if (j & (1 << KB)) continue;
            const int j1 = j | (1 << KB);
            const amp_t<T> a0 = a[j], a1 = a[j1], l0 = l[j], l1 = l[j1];
            // Im <lambda| Y |phi> over the pair: Re(conj(l1) a0) - Re(conj(l0) a1)
            pv[q++] = (l1.x * a0.x + l1.y * a0.y) - (l0.x * a1.x + l0.y * a1.y);
            // RY^dagger = [[c, s], [-s, c]]
            a[j] = mk<T>(c * a0.x + s * a1.x, c * a0.y + s * a1.y);
            a[j1] = mk<T>(c * a1.x - s * a0.x, c * a1.y - s * a0.y);
            l[j] = mk<T>(c * l0.x + s * l1.x, c * l0.y + s * l1.y);
            l[j1] = mk<T>(c * l1.x - s * l0.x, c * l1.y - s * l0.y);
        }
        return tree_sum<NA / 2, T>(pv);
    }
}

template <int KB, int NA, typename T>
VQG_DEV T rev_rx(amp_t<T> (&a)[NA], amp_t<T> (&l)[NA], const Mat2<T> &ud) {
    T pv[NA / 2];
    int q = 0;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        const int j1 = j | (1 << KB);
        const amp_t<T> a0 = a[j], a1 = a[j1], l0 = l[j], l1 = l[j1];
        // Im <lambda| X |phi>: Im(conj(l0) a1) + Im(conj(l1) a0)
        pv[q++] = (l0.x * a1.y - l0.y * a1.x) + (l1.x * a0.y - l1.y * a0.x);
        apply2<T>(ud, a[j], a[j1]);
        apply2<T>(ud, l[j], l[j1]);
    }
    return tree_sum<NA / 2, T>(pv);
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

// Controlled 2x2 in reverse (App. A: the derivative of C_c[U] is dU projected onto
// control = 1, so only pairs with the control set contribute).  G selects the value:
// 0: Im<l|X|phi>, 1: Im<l|Y|phi>, 2: Im<l|Z|phi> (controlled rotations, as for RX/RY/RZ);
// 3: -2 Im(conj(l1) phi1) (phase gates: dP/dt = i e^{it}|1><1|).
template <int G, int KB, int NA, typename T>
VQG_DEV T rev_cgen(amp_t<T> (&a)[NA], amp_t<T> (&l)[NA], const Mat2<T> &ud, uint32_t rc, bool thr_c) {
    T v = 0;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (j & (1 << KB)) continue;
        const bool c = rc ? ((j & rc) != 0) : thr_c;
        if (!c) continue;
        const int j1 = j | (1 << KB);
        const amp_t<T> a0 = a[j], a1 = a[j1], l0 = l[j], l1 = l[j1];
        if constexpr (G == 0) v += (l0.x * a1.y - l0.y * a1.x) + (l1.x * a0.y - l1.y * a0.x);
        else if constexpr (G == 1) v += (l1.x * a0.x + l1.y * a0.y) - (l0.x * a1.x + l0.y * a1.y);
        else if constexpr (G == 2) v += (l0.x * a0.y - l0.y * a0.x) - (l1.x * a1.y - l1.y * a1.x);
        else v += (T)-2 * (l1.x * a1.y - l1.y * a1.x);
        apply2<T>(ud, a[j], a[j1]);
        apply2<T>(ud, l[j], l[j1]);
    }
    return v;
}

// Reverse diagonal block.  Every RZ of the block gets Im <lambda| Z_q |phi> from the
// block's input pair: the other gates of the block are diagonal, commute with Z_q and
// cancel between bra and ket.  With p_j = Im(conj(lambda_j) phi_j), an RZ on register
// bit k needs sum_j (-1)^{j_k} p_j and an RZ on a thread-level qubit +-sum_j p_j.
template <int R, int NA, typename T>
VQG_DEV void rev_diag(amp_t<T> (&a)[NA], amp_t<T> (&l)[NA], const Prog<T, R> &pg, const FDiag &D,
                      int di, uint64_t gb, T *stash_row, int nt, amp_t<T> &phase, T k2acc) {
    if (D.n_rz > 0) {
        T H[R], S;
        if constexpr (std::is_same<T, float>::value) {
            // p_j = Im(conj(l_j) a_j) held as pairs q_m = (p_2m, p_2m+1): every fold of the
            // tree below is one packed add for two index-bit-0 lanes; the lanes meet only
            // in the final scalar adds.
            float2 q[NA / 2];
#pragma unroll
            for (int m = 0; m < NA / 2; ++m)
                q[m] = make_float2(l[2 * m].x * a[2 * m].y - l[2 * m].y * a[2 * m].x,
                                   l[2 * m + 1].x * a[2 * m + 1].y - l[2 * m + 1].y * a[2 * m + 1].x);
#pragma unroll
            for (int k = 1; k < R; ++k) {  // fold index bit k (bit k - 1 of m)
                const int len = (NA / 2) >> (k - 1);
                float2 h = q[0];
#pragma unroll
                for (int m = 1; m < len / 2; ++m) h = __fadd2_rn(h, q[2 * m]);
                H[k] = h.x + h.y;
#pragma unroll
                for (int m = 0; m < len / 2; ++m) q[m] = __fadd2_rn(q[2 * m], q[2 * m + 1]);
            }
            H[0] = q[0].x;
            S = q[0].x + q[0].y;
        } else {
            T p[NA];
#pragma unroll
            for (int j = 0; j < NA; ++j) p[j] = l[j].x * a[j].y - l[j].y * a[j].x;
            // H[k] = sum over register index bit k = 0, S = sum of all, from one pairwise
            // tree: level k folds bit k, and H[k] sums the bit-k = 0 entries of the level's
            // input (2^R - 1 + sum_k (2^(R-1-k) - 1) adds instead of R (2^(R-1) - 1) + 2^R - 1)
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const int len = NA >> k;
                T h[NA / 2];
#pragma unroll
                for (int m = 0; m < len / 2; ++m) h[m] = p[2 * m];
                H[k] = tree_sum<NA / 2, T>(h, len / 2);
#pragma unroll
                for (int m = 0; m < len / 2; ++m) p[m] = p[2 * m] + p[2 * m + 1];
            }
            S = p[0];
        }
        const int i0 = D.item0 - pg.item_base;
        T v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            v[r] = 0;
            if (r < D.n_rz) {
                const FDItem &x = pg.it[i0 + r];
                if (x.type == DI_RZ_REG) {
                    T h = H[0];
#pragma unroll
                    for (int k = 1; k < R; ++k)
                        if (x.k0 == k) h = H[k];
                    v[r] = (T)2 * h - S;  // sum over bit 0 minus sum over bit 1
                } else {
                    v[r] = (gb & x.g0) ? -S : S;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (r < D.n_rz) {
                if constexpr (std::is_same<T, float>::value) v[r] *= k2acc;  // the stage's scale so far
                stash_row[r * nt] = v[r];
            }
    }
    amp_t<T> tau;
    uint32_t c;
    diag_thread<T, R>(pg, D, gb, tau, c);
    phase = cmul<T>(tau, phase);  // common to phi and lambda: leaves every reduction unchanged
    const amp_t<T> *tab = pg.tab + di * NA;
    const uint32_t w = walsh_bits(c);
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        amp_t<T> d = tab[j];
        if ((w >> j) & 1u) d = neg<T>(d);
        if constexpr (std::is_same<T, float>::value) {
            // packed FP32 pairs; the factor's broadcasts serve phi and lambda:
            // d z = (d.x, d.x) * z + (-d.y, d.y) * (z.y, z.x)
            const float2 dr = make_float2(d.x, d.x), di2 = make_float2(-d.y, d.y);
            a[j] = __ffma2_rn(dr, a[j], __fmul2_rn(di2, make_float2(a[j].y, a[j].x)));
            l[j] = __ffma2_rn(dr, l[j], __fmul2_rn(di2, make_float2(l[j].y, l[j].x)));
        } else {
            a[j] = cmul<T>(d, a[j]);
            l[j] = cmul<T>(d, l[j]);
        }
    }
}

// ------------------------------------------------------------------ tile I/O
template <typename T, int K>
struct TileIO {
    static constexpr int L = FT<T>::L, AB = FT<T>::AB;
    static constexpr int TILE = 1 << K, ROWS = 1 << (K - L);
    static constexpr int CA = 16 / AB;          // amplitudes per 16-byte chunk
    static constexpr int CPR = (1 << L) / CA;   // chunks per 128-byte row
    static constexpr int CHUNKS = TILE / CA;

    // Thread tid moves chunks c = tid + NT*i.  Their rows are tid/CPR + (NT/CPR)*i and
    // their column tid%CPR, so the shared-memory slot is swz(t0) ^ swz(i << SHI) (swz is
    // linear) and the row offset row_off[row0] | row_off[(NT/CPR)*i] (the deposit of
    // disjoint bits is linear too): one XOR per chunk instead of a full recomputation.
    template <int NT>
    struct Geo {
        static_assert(NT % CPR == 0 && CHUNKS % NT == 0, "chunk geometry");
        static constexpr int CPT = CHUNKS / NT, RSTEP = NT / CPR;
        static constexpr int SHI = L + (RSTEP == 1 ? 0 : RSTEP == 2 ? 1 : RSTEP == 4 ? 2 : RSTEP == 8 ? 3 :
                                        RSTEP == 16 ? 4 : RSTEP == 32 ? 5 : RSTEP == 64 ? 6 : 7);
    };

    // L2ONLY: bypass L1 (needed when another block of the same launch wrote the data).
    // zmask: index bits on which the source is known to be zero (FPass::zero_in): such
    // amplitudes are not read (the memory there need not hold zeros) and enter as zero.
    template <int NT, bool L2ONLY = false>
    static VQG_DEV void load(amp_t<T> *tile, const amp_t<T> *__restrict__ src, uint64_t base,
                             const uint64_t *row_off, int tid, uint64_t zmask = 0) {
        using G = Geo<NT>;
        const int row0 = tid / CPR, col = tid % CPR;
        const uint32_t s0 = swz<AB>((uint32_t)(row0 << L) | (uint32_t)(col * CA));
        const uint64_t o0 = (base | row_off[row0]) + col * CA;
        const amp_t<T> *g0 = src + o0;
        float4 v[G::CPT];  // every global load in flight before the first shared store
#pragma unroll
        for (int i = 0; i < G::CPT; ++i) {
            const float4 *g = reinterpret_cast<const float4 *>(g0 + row_off[G::RSTEP * i]);
            if ((o0 | row_off[G::RSTEP * i]) & zmask) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            else v[i] = L2ONLY ? __ldcg(g) : __ldcs(g);
            if (CA == 2 && (zmask & 1ull)) v[i].z = v[i].w = 0.f;  // the chunk's odd amplitude
        }
#pragma unroll
        for (int i = 0; i < G::CPT; ++i) put_chunk(tile, s0 ^ swz<AB>((uint32_t)i << G::SHI), v[i]);
    }
    // Two tiles at the same positions (the reverse pass's phi and lambda): every global
    // load of both is issued before the first shared-memory store.
    template <int NT, bool L2ONLY = false>
    static VQG_DEV void load2(amp_t<T> *ta, const amp_t<T> *__restrict__ sa, amp_t<T> *tb,
                              const amp_t<T> *__restrict__ sb, uint64_t base, const uint64_t *row_off, int tid) {
        using G = Geo<NT>;
        const int row0 = tid / CPR, col = tid % CPR;
        const uint32_t s0 = swz<AB>((uint32_t)(row0 << L) | (uint32_t)(col * CA));
        const uint64_t o0 = (base | row_off[row0]) + col * CA;
        float4 va[G::CPT], vb[G::CPT];
#pragma unroll
        for (int i = 0; i < G::CPT; ++i) {
            const uint64_t o = o0 + row_off[G::RSTEP * i];
            const float4 *ga = reinterpret_cast<const float4 *>(sa + o);
            const float4 *gb = reinterpret_cast<const float4 *>(sb + o);
            va[i] = L2ONLY ? __ldcg(ga) : __ldcs(ga);
            vb[i] = L2ONLY ? __ldcg(gb) : __ldcs(gb);
        }
#pragma unroll
        for (int i = 0; i < G::CPT; ++i) {
            put_chunk(ta, s0 ^ swz<AB>((uint32_t)i << G::SHI), va[i]);
            put_chunk(tb, s0 ^ swz<AB>((uint32_t)i << G::SHI), vb[i]);
        }
    }
    // Ask L2 for the rows of a tile (one 128-byte row = one L2 line per request) one tile
    // ahead of its load: the load then hits L2 instead of waiting on HBM.
    template <int NT>
    static VQG_DEV void prefetch(const amp_t<T> *src, uint64_t base, const uint64_t *row_off, int tid,
                                 uint64_t zmask = 0) {
        for (int r = tid; r < ROWS; r += NT) {
            if ((base | row_off[r]) & zmask & ~(uint64_t)((1 << L) - 1)) continue;  // a row known zero
            const amp_t<T> *p = src + (base | row_off[r]);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
        }
    }
    template <int NT>
    static VQG_DEV void zero(amp_t<T> *tile, uint64_t base, int tid) {
        using G = Geo<NT>;
        const int row0 = tid / CPR, col = tid % CPR;
        const uint32_t s0 = swz<AB>((uint32_t)(row0 << L) | (uint32_t)(col * CA));
#pragma unroll
        for (int i = 0; i < G::CPT; ++i) put_chunk(tile, s0 ^ swz<AB>((uint32_t)i << G::SHI), make_float4(0.f, 0.f, 0.f, 0.f));
        if (base == 0 && tid == 0) tile[swz<AB>(0)] = mk<T>((T)1, (T)0);
    }
    // A 16-byte global chunk <-> its CA amplitudes in the tile arithmetic (float-float
    // amplitudes are FP64 in memory).
    static VQG_DEV void unpack(float4 v, amp_t<T> *a) {
        if constexpr (AB == 8) {
            a[0] = mk<T>(v.x, v.y);
            a[1] = mk<T>(v.z, v.w);
        } else if constexpr (FT<T>::conv) {
            union {
                float4 f;
                double2 d;
            } u;
            u.f = v;
            a[0] = mk<T>(T(u.d.x), T(u.d.y));
        } else {
            union {
                float4 f;
                amp_t<T> a;
            } u;
            u.f = v;
            a[0] = u.a;
        }
    }
    static VQG_DEV float4 pack(const amp_t<T> *a) {
        if constexpr (AB == 8) {
            return make_float4(a[0].x, a[0].y, a[1].x, a[1].y);
        } else {
            union {
                float4 f;
                double2 d;
            } u;
            u.d = make_double2((double)a[0].x, (double)a[0].y);
            return u.f;
        }
    }
    // A 16-byte chunk (two complex64 or one complex128 amplitudes) at swizzled slot s of its
    // first amplitude.  For complex64 the second amplitude sits at s ^ swz(1) = s ^ 1.
    static VQG_DEV void put_chunk(amp_t<T> *tile, uint32_t s, float4 v) {
        if constexpr (AB == 8 || FT<T>::conv) {
            amp_t<T> a[CA];
            unpack(v, a);
            tile[s] = a[0];
            if constexpr (CA == 2) tile[s ^ 1u] = a[1];
        } else {
            *reinterpret_cast<float4 *>(tile + s) = v;
        }
    }
    static VQG_DEV float4 get_chunk(const amp_t<T> *tile, uint32_t s) {
        if constexpr (AB == 8) {
            const amp_t<T> a[2] = {tile[s], tile[s ^ 1u]};
            return pack(a);
        } else if constexpr (FT<T>::conv) {
            return pack(tile + s);
        } else {
            return *reinterpret_cast<const float4 *>(tile + s);
        }
    }
    template <int NT>
    static VQG_DEV void store(const amp_t<T> *tile, amp_t<T> *__restrict__ dst, uint64_t base,
                              const uint64_t *row_off, int tid) {
        using G = Geo<NT>;
        const int row0 = tid / CPR, col = tid % CPR;
        const uint32_t s0 = swz<AB>((uint32_t)(row0 << L) | (uint32_t)(col * CA));
        amp_t<T> *g0 = dst + ((base | row_off[row0]) + col * CA);
        float4 v[G::CPT];  // every shared load before the first global store
#pragma unroll
        for (int i = 0; i < G::CPT; ++i) v[i] = get_chunk(tile, s0 ^ swz<AB>((uint32_t)i << G::SHI));
#pragma unroll
        for (int i = 0; i < G::CPT; ++i) __stcs(reinterpret_cast<float4 *>(g0 + row_off[G::RSTEP * i]), v[i]);
    }
    // Zeros at a tile's positions in global memory (a tile that holds no amplitude).
    template <int NT>
    static VQG_DEV void store_zero(amp_t<T> *__restrict__ dst, uint64_t base, const uint64_t *row_off, int tid) {
        using G = Geo<NT>;
        const int row0 = tid / CPR, col = tid % CPR;
        amp_t<T> *g0 = dst + ((base | row_off[row0]) + col * CA);
#pragma unroll
        for (int i = 0; i < G::CPT; ++i)
            __stcs(reinterpret_cast<float4 *>(g0 + row_off[G::RSTEP * i]), make_float4(0.f, 0.f, 0.f, 0.f));
    }
};

VQG_DEV uint64_t tile_base(uint64_t tile, const int32_t *nontile, int n_nontile) {
    uint64_t b = 0;
    for (int i = 0; i < n_nontile; ++i) b |= ((tile >> i) & 1ull) << nontile[i];
    return b;
}

template <typename T, int K>
VQG_DEV void fill_row_offsets(const int32_t *high, uint64_t *row_off, int tid, int nt) {
    constexpr int L = FT<T>::L, ROWS = 1 << (K - L);
    for (int r = tid; r < ROWS; r += nt) {
        uint64_t off = 0;
        for (int i = 0; i < K - L; ++i)
            if ((r >> i) & 1) off |= 1ull << high[i];
        row_off[r] = off;
    }
}

// Tile-local smem base and global index of register index 0 for this thread.
template <int K, int R, int AB>
VQG_DEV void thread_base(const FStage &st, int tid, uint64_t base, uint32_t &sb, uint64_t &gb) {
    sb = 0;
    gb = base;
#pragma unroll
    for (int b = 0; b < K - R; ++b)
        if ((tid >> b) & 1) sb ^= st.thr_sw[b], gb |= 1ull << st.thr_q[b];
}

template <int R, int NA>
VQG_DEV uint32_t reg_addr(uint32_t sb, const uint32_t (&w)[R], int j) {
    uint32_t ad = sb;
#pragma unroll
    for (int k = 0; k < R; ++k)
        if ((j >> k) & 1) ad ^= w[k];
    return ad;
}

// ------------------------------------------------------------------ per-tile bodies
// One tile of a forward pass: load (or |0...0>), run the stages, store.
template <typename T, int K, int R, bool L2ONLY>
VQG_DEV void fwd_tile(amp_t<T> *tile, const uint64_t *row_off, const Prog<T, R> &pg, int n_stage,
                      uint64_t base, bool from_zero, const amp_t<T> *__restrict__ src,
                      amp_t<T> *__restrict__ dst, int tid, uint64_t zmask = 0) {
    using A = amp_t<T>;
    using IO = TileIO<T, K>;
    constexpr int AB = FT<T>::AB, NT = 1 << (K - R), NA = 1 << R;
    if (from_zero) IO::template zero<NT>(tile, base, tid);
    else IO::template load<NT, L2ONLY>(tile, src, base, row_off, tid, zmask);
    __syncthreads();
    for (int s = 0; s < n_stage; ++s) {
        const FStage &st = pg.st[s];
        uint32_t sb;
        uint64_t gb;
        thread_base<K, R, AB>(st, tid, base, sb, gb);
        uint32_t w[R];
#pragma unroll
        for (int k = 0; k < R; ++k) w[k] = st.reg_sw[k];
        A a[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) a[j] = tile[reg_addr<R, NA>(sb, w, j)];
        A phase = mk<T>((T)1, (T)0);
        T kacc = (T)1;  // product K of the k of the stage's scaled RY ops (complex64)
        const int o0 = st.op0 - pg.op_base;
        for (int o = o0; o < o0 + st.n_op; ++o) apply_fwd_op<R, NA, T>(a, pg, o, gb, phase, kacc);
        asm volatile("" : "+r"(sb));  // recompute the addresses instead of keeping them live
        if (st.has_phase) {
            if constexpr (std::is_same<T, float>::value) phase = mk<T>(phase.x * kacc, phase.y * kacc);
#pragma unroll
            for (int j = 0; j < NA; ++j) tile[reg_addr<R, NA>(sb, w, j)] = cmul<T>(phase, a[j]);
        } else if (scaled_stage<T>(kacc)) {
            if constexpr (std::is_same<T, float>::value) {
                const float2 sv = make_float2(kacc, kacc);
#pragma unroll
                for (int j = 0; j < NA; ++j) tile[reg_addr<R, NA>(sb, w, j)] = __fmul2_rn(sv, a[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < NA; ++j) tile[reg_addr<R, NA>(sb, w, j)] = a[j];
        }
        __syncthreads();
    }
    IO::template store<NT>(tile, dst, base, row_off, tid);
    __syncthreads();
}

// Reduce stash rows (per-thread partials) into the per-slot FP64 accumulators: row r goes
// to slot first + r.  One warp per row, lanes sum NT/32 partials each (16-byte loads
// where NT allows), then the 32-lane tree; fixed order, so results are reproducible.
template <typename T, int NT>
VQG_DEV void reduce_rows(const T *stash, int first, int count, double *acc, int tid) {
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int V = 16 / sizeof(T);  // values per 16-byte load
    for (int r = warp; r < count; r += NT / 32) {
        T v = 0;
        if constexpr (NT % (32 * V) != 0 || FT<T>::conv) {
            for (int i = lane; i < NT; i += 32) v += stash[r * NT + i];
        } else {
#pragma unroll
            for (int i = lane * V; i < NT; i += 32 * V) {
                const float4 q = *reinterpret_cast<const float4 *>(stash + r * NT + i);
                if constexpr (sizeof(T) == 4) v += (q.x + q.y) + (q.z + q.w);
                else {
                    const double2 d = *reinterpret_cast<const double2 *>(&q);
                    v += d.x + d.y;
                }
            }
        }
        v = warp_tree<T>(v);
        if (lane == 0) acc[first + r] += (double)v;
    }
}

// The rows of a stage's last stash segment (their local slots are contiguous).
template <typename T, int NT>
VQG_DEV void reduce_stash(const T *stash, const FStage &st, double *acc, int tid) {
    reduce_rows<T, NT>(stash, st.row_slot[0], st.n_rows, acc, tid);
}

template <typename T> constexpr int stash_rows() { return sizeof(T) == 4 ? kMaxStageRows : kMaxStageRowsDbl; }

// Per-thread geometry of one register stage: shared-memory slot sb and global index gb of
// register index 0, and the swizzled offsets of the register bits.
template <typename T, int K, int R>
struct StageGeo {
    uint32_t sb;
    uint64_t gb;
    uint32_t w[R];
    VQG_DEV void init(const FStage &st, int tid, uint64_t base) {
        thread_base<K, R, FT<T>::AB>(st, tid, base, sb, gb);
#pragma unroll
        for (int k = 0; k < R; ++k) w[k] = st.reg_sw[k];
    }
};

// Reverse op bodies, shared by the interpreted tile pass and the per-pass specialised
// kernels.  Each returns the thread's partial of the op's reduction value (stored by the
// caller in the op's stash row) where the op has one; m is the op's parameter row.
template <int KB, int R, typename T>
VQG_DEV T rev_op_ry(amp_t<T> (&a)[1 << R], amp_t<T> (&l)[1 << R], const amp_t<T> *m, T &kacc, T &k2acc) {
    constexpr int NA = 1 << R;
    T v1;
    if constexpr (std::is_same<T, float>::value) {  // scaled form (see load_prog)
        const float2 p1 = m[1], p2 = m[2];
        v1 = rev_ry_scaled<KB, NA>(a, l, p1.x, p1.y != 0.f);
        v1 *= k2acc;  // the inputs held the true values divided by K so far
        kacc *= p2.x;
        k2acc *= p2.y;
    } else {
        const amp_t<T> cs = m[0];
        v1 = rev_ry<KB, NA, T>(a, l, cs.x, cs.y);
    }
    return v1;
}
template <int KB, int R, typename T>
VQG_DEV T rev_op_rx(amp_t<T> (&a)[1 << R], amp_t<T> (&l)[1 << R], const amp_t<T> *m, T k2acc) {
    const Mat2<T> ud = dagger<T>(mat_of<T>(m));
    T v1 = rev_rx<KB, 1 << R, T>(a, l, ud);
    if constexpr (std::is_same<T, float>::value) v1 *= k2acc;
    return v1;
}
// U3: eight values, stored in stash rows row .. row + 7 (srow points at row, stride nt)
template <int KB, int R, typename T>
VQG_DEV void rev_op_u3(amp_t<T> (&a)[1 << R], amp_t<T> (&l)[1 << R], const amp_t<T> *m, T k2acc, T *srow, int nt) {
    const Mat2<T> ud = dagger<T>(mat_of<T>(m));
    T v8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    rev_u3<KB, 1 << R, T>(a, l, ud, v8);
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        if constexpr (std::is_same<T, float>::value) v8[x] *= k2acc;
        srow[x * nt] = v8[x];
    }
}
template <int KB, int R, typename T>
VQG_DEV void rev_op_cnot(amp_t<T> (&a)[1 << R], amp_t<T> (&l)[1 << R], uint32_t rm0, bool thr_c) {
    op_cnot<KB, 1 << R, T>(a, rm0, thr_c);
    op_cnot<KB, 1 << R, T>(l, rm0, thr_c);
}
// controlled rotations (G = 0, 1, 2: X, Y, Z generator) and phase gates (G = 3)
template <int G, int KB, int R, typename T>
VQG_DEV T rev_op_cgen(amp_t<T> (&a)[1 << R], amp_t<T> (&l)[1 << R], const amp_t<T> *m, uint32_t rm0, bool thr_c,
                      T k2acc) {
    const Mat2<T> ud = dagger<T>(mat_of<T>(m));
    T v1 = rev_cgen<G, KB, 1 << R, T>(a, l, ud, rm0, thr_c);
    if constexpr (std::is_same<T, float>::value) v1 *= k2acc;
    return v1;
}

template <typename T, int K, int R>
VQG_DEV void rev_gather(const StageGeo<T, K, R> &g, const amp_t<T> *tphi, const amp_t<T> *tlam,
                        amp_t<T> (&a)[1 << R], amp_t<T> (&l)[1 << R]) {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        const uint32_t ad = reg_addr<R, 1 << R>(g.sb, g.w, j);
        a[j] = tphi[ad];
        l[j] = tlam[ad];
    }
}

// Write the stage's amplitudes back: multiplied by the stage's per-thread phase (which
// also carries the scaled-RY factor K) or by K alone, or as they are.
template <typename T, int K, int R>
VQG_DEV void rev_scatter(StageGeo<T, K, R> &g, bool has_phase, amp_t<T> *tphi, amp_t<T> *tlam,
                         const amp_t<T> (&a)[1 << R], const amp_t<T> (&l)[1 << R], amp_t<T> phase, T kacc) {
    constexpr int NA = 1 << R;
    asm volatile("" : "+r"(g.sb));  // recompute the addresses instead of keeping them live
    if (has_phase) {
        if constexpr (std::is_same<T, float>::value) {  // packed, broadcasts shared by both states
            phase = mk<T>(phase.x * kacc, phase.y * kacc);
            const float2 pr = make_float2(phase.x, phase.x), pi2 = make_float2(-phase.y, phase.y);
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                const uint32_t ad = reg_addr<R, NA>(g.sb, g.w, j);
                tphi[ad] = __ffma2_rn(pr, a[j], __fmul2_rn(pi2, make_float2(a[j].y, a[j].x)));
                tlam[ad] = __ffma2_rn(pr, l[j], __fmul2_rn(pi2, make_float2(l[j].y, l[j].x)));
            }
        } else {
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                const uint32_t ad = reg_addr<R, NA>(g.sb, g.w, j);
                tphi[ad] = cmul<T>(phase, a[j]);
                tlam[ad] = cmul<T>(phase, l[j]);
            }
        }
    } else if (scaled_stage<T>(kacc)) {
        if constexpr (std::is_same<T, float>::value) {
            const float2 sv = make_float2(kacc, kacc);
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                const uint32_t ad = reg_addr<R, NA>(g.sb, g.w, j);
                tphi[ad] = __fmul2_rn(sv, a[j]);
                tlam[ad] = __fmul2_rn(sv, l[j]);
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const uint32_t ad = reg_addr<R, NA>(g.sb, g.w, j);
            tphi[ad] = a[j];
            tlam[ad] = l[j];
        }
    }
}

// One tile of a reverse pass.  Each op stores its per-thread FP32 partial(s) in the
// stage's stash rows (no cross-lane dependency in the op loop); after the stage the
// rows are reduced into acc (FP64, one value per local slot).
template <typename T, int K, int R, bool L2ONLY>
VQG_DEV void rev_tile(amp_t<T> *tphi, amp_t<T> *tlam, const uint64_t *row_off, const Prog<T, R> &pg,
                      int n_stage, uint64_t base, const amp_t<T> *__restrict__ phi_src,
                      amp_t<T> *__restrict__ phi_dst, amp_t<T> *__restrict__ lam, double *acc,
                      T *stash, int tid, bool write_phi = true, bool write_lam = true) {
    using A = amp_t<T>;
    using IO = TileIO<T, K>;
    constexpr int AB = FT<T>::AB, NT = 1 << (K - R), NA = 1 << R;
    IO::template load2<NT, L2ONLY>(tphi, phi_src, tlam, lam, base, row_off, tid);
    __syncthreads();
    for (int s = 0; s < n_stage; ++s) {
        const FStage &st = pg.st[s];
        uint32_t sb;
        uint64_t gb;
        thread_base<K, R, AB>(st, tid, base, sb, gb);
        uint32_t w[R];
#pragma unroll
        for (int k = 0; k < R; ++k) w[k] = st.reg_sw[k];
        A a[NA], l[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const uint32_t ad = reg_addr<R, NA>(sb, w, j);
            a[j] = tphi[ad];
            l[j] = tlam[ad];
        }
        A phase = mk<T>((T)1, (T)0);
        // complex64: the scaled RY ops leave phi and lambda holding their true values
        // divided by K, the product of the ops' k: kacc = K (multiplied back at the scatter),
        // k2acc = K^2 (multiplies every reduction partial formed from the held values)
        T kacc = (T)1, k2acc = (T)1;
        const int o0 = st.op0 - pg.op_base;
        for (int o = o0; o < o0 + st.n_op; ++o) {
            const FOp op = pg.op[o];
            const A *m = pg.prm + 4 * o;
            T v1 = 0;
            bool red1 = false;
            switch (op.type) {
            case OP_RY: {
                if constexpr (std::is_same<T, float>::value) {  // scaled form (see load_prog)
                    const float2 p1 = m[1], p2 = m[2];
                    with_k<R>(op.k, [&](auto kb) {
                        v1 = rev_ry_scaled<decltype(kb)::value, NA>(a, l, p1.x, p1.y != 0.f);
                    });
                    v1 *= k2acc;  // the inputs held the true values divided by K so far
                    kacc *= p2.x;
                    k2acc *= p2.y;
                } else {
                    const A cs = m[0];
                    with_k<R>(op.k, [&](auto kb) { v1 = rev_ry<decltype(kb)::value, NA, T>(a, l, cs.x, cs.y); });
                }
                red1 = true;
                break;
            }
            case OP_RX: {
                const Mat2<T> ud = dagger<T>(mat_of<T>(m));
                with_k<R>(op.k, [&](auto kb) { v1 = rev_rx<decltype(kb)::value, NA, T>(a, l, ud); });
                if constexpr (std::is_same<T, float>::value) v1 *= k2acc;
                red1 = true;
                break;
            }
            case OP_U3: {
                const Mat2<T> ud = dagger<T>(mat_of<T>(m));
                T v8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                with_k<R>(op.k, [&](auto kb) { rev_u3<decltype(kb)::value, NA, T>(a, l, ud, v8); });
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    if constexpr (std::is_same<T, float>::value) v8[x] *= k2acc;
                    stash[(op.row + x) * NT + tid] = v8[x];
                }
                break;
            }
            case OP_CNOT: {
                const bool c = op.rm0 ? false : ((gb >> op.cq) & 1ull) != 0;
                with_k<R>(op.k, [&](auto kb) {
                    op_cnot<decltype(kb)::value, NA, T>(a, op.rm0, c);
                    op_cnot<decltype(kb)::value, NA, T>(l, op.rm0, c);
                });
                break;
            }
            case OP_CRX:
            case OP_CRY:
            case OP_CRZ:
            case OP_PH: {
                const Mat2<T> ud = dagger<T>(mat_of<T>(m));
                const bool c = thread_control(op, gb);
                with_k<R>(op.k, [&](auto kb) {
                    constexpr int KB = decltype(kb)::value;
                    if (op.type == OP_CRX) v1 = rev_cgen<0, KB, NA, T>(a, l, ud, op.rm0, c);
                    else if (op.type == OP_CRY) v1 = rev_cgen<1, KB, NA, T>(a, l, ud, op.rm0, c);
                    else if (op.type == OP_CRZ) v1 = rev_cgen<2, KB, NA, T>(a, l, ud, op.rm0, c);
                    else v1 = rev_cgen<3, KB, NA, T>(a, l, ud, op.rm0, c);
                });
                if constexpr (std::is_same<T, float>::value) v1 *= k2acc;
                red1 = true;
                break;
            }
            case OP_DIAG:
                rev_diag<R, NA, T>(a, l, pg, pg.dg[op.diag], op.diag, gb, stash + op.row * NT + tid, NT, phase,
                                   k2acc);
                break;
            case OP_FLUSH:  // uniform: every thread runs the same op list
                __syncthreads();
                reduce_rows<T, NT>(stash, op.lslot, op.row, acc, tid);
                __syncthreads();
                break;
            default:
                break;
            }
            if (red1) stash[op.row * NT + tid] = v1;
        }
        asm volatile("" : "+r"(sb));  // recompute the addresses instead of keeping them live
        if (st.has_phase) {
            if constexpr (std::is_same<T, float>::value) {  // packed, broadcasts shared by both states
                phase = mk<T>(phase.x * kacc, phase.y * kacc);
                const float2 pr = make_float2(phase.x, phase.x), pi2 = make_float2(-phase.y, phase.y);
#pragma unroll
                for (int j = 0; j < NA; ++j) {
                    const uint32_t ad = reg_addr<R, NA>(sb, w, j);
                    tphi[ad] = __ffma2_rn(pr, a[j], __fmul2_rn(pi2, make_float2(a[j].y, a[j].x)));
                    tlam[ad] = __ffma2_rn(pr, l[j], __fmul2_rn(pi2, make_float2(l[j].y, l[j].x)));
                }
            } else {
#pragma unroll
                for (int j = 0; j < NA; ++j) {
                    const uint32_t ad = reg_addr<R, NA>(sb, w, j);
                    tphi[ad] = cmul<T>(phase, a[j]);
                    tlam[ad] = cmul<T>(phase, l[j]);
                }
            }
        } else if (scaled_stage<T>(kacc)) {
            if constexpr (std::is_same<T, float>::value) {
                const float2 sv = make_float2(kacc, kacc);
#pragma unroll
                for (int j = 0; j < NA; ++j) {
                    const uint32_t ad = reg_addr<R, NA>(sb, w, j);
                    tphi[ad] = __fmul2_rn(sv, a[j]);
                    tlam[ad] = __fmul2_rn(sv, l[j]);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                const uint32_t ad = reg_addr<R, NA>(sb, w, j);
                tphi[ad] = a[j];
                tlam[ad] = l[j];
            }
        }
        __syncthreads();
        if (st.n_rows) {
            reduce_stash<T, NT>(stash, st, acc, tid);
            __syncthreads();
        }
    }
    if (write_phi) IO::template store<NT>(tphi, phi_dst, base, row_off, tid);
    if (write_lam) IO::template store<NT>(tlam, lam, base, row_off, tid);
    __syncthreads();
}

// ------------------------------------------------------------------ forward pass
template <typename T, int K, int R, typename CAPS = FullCaps>
struct FwdCfg {
    using Caps = CAPS;
    static constexpr int NT = 1 << (K - R);
    static constexpr size_t o_row = (size_t)(1 << K) * FT<T>::AB;
    static constexpr size_t o_prog = o_row + sizeof(uint64_t) * (1 << (K - FT<T>::L));
    static constexpr size_t prog_bytes = Prog<T, R>::template Layout<CAPS>::bytes;
    static constexpr size_t smem() { return o_prog + prog_bytes; }
    static_assert(o_prog + prog_bytes <= 227 * 1024, "forward pass exceeds shared memory");
};

template <typename T, int K, int R>
__global__ void __launch_bounds__(1 << (K - R), (1 << (K - R)) >= 512 ? 1 : 2)
    k_fused_fwd(const amp_t<T> *__restrict__ src, amp_t<T> *__restrict__ dst,
                const FPass *__restrict__ passes, int pi, const FStage *__restrict__ stages,
                const FOp *__restrict__ ops, const FDiag *__restrict__ diags,
                const FDItem *__restrict__ items, const typename FT<T>::mat_t *__restrict__ mats, uint64_t n_tiles) {
    using A = amp_t<T>;
    using C = FwdCfg<T, K, R>;
    constexpr int NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem[];
    A *tile = reinterpret_cast<A *>(smem);
    uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + C::o_row);
    Prog<T, R> pg;
    pg.template bind<typename C::Caps>(smem + C::o_prog);
    const FPass &P = passes[pi];
    const int tid = threadIdx.x;
    fill_row_offsets<T, K>(P.high, row_off, tid, NT);
    load_prog<T, R>(pg, P.stage0, P.n_stage, P.diag0, P.n_diag, stages, ops, diags, items, mats, false, tid, NT);
    __syncthreads();
    const uint64_t n_act = 1ull << P.n_active;  // later tiles hold zeros only (FPass::n_active)
    for (uint64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        if (ti >= n_act) {
            TileIO<T, K>::template store_zero<NT>(dst, tile_base(ti, P.nontile, P.n_nontile), row_off, tid);
            continue;
        }
        if (ti + gridDim.x < n_act && !P.from_zero)
            TileIO<T, K>::template prefetch<NT>(src, tile_base(ti + gridDim.x, P.nontile, P.n_nontile), row_off, tid,
                                                P.zero_in);
        fwd_tile<T, K, R, false>(tile, row_off, pg, P.n_stage, tile_base(ti, P.nontile, P.n_nontile),
                                 P.from_zero != 0, src, dst, tid, P.zero_in);
    }
}

// ------------------------------------------------------------------ reverse pass
// Shared-memory layout of a reverse pass: phi and lambda tiles, row offsets, the program,
// FP64 accumulators, ROWS stash rows of NT values and the slot map.  Host code sizes the
// specialised kernels (pass-sized programs, ROWS = two stash buffers) with rev_offsets.
struct RevOffsets {
    size_t row, prog, acc, stash, map, bytes;
};
__host__ __device__ constexpr RevOffsets rev_offsets(int K, int R, int L, size_t ab, size_t tsize, size_t prog_bytes,
                                                     int rows) {
    RevOffsets o{};
    o.row = 2 * ((size_t)1 << K) * ab;
    o.prog = o.row + sizeof(uint64_t) * ((size_t)1 << (K - L));
    o.acc = o.prog + prog_bytes;
    o.stash = o.acc + sizeof(double) * kMaxPassSlots;
    o.map = o.stash + tsize * (size_t)rows * ((size_t)1 << (K - R));
    o.bytes = o.map + sizeof(int) * kMaxPassSlots;
    return o;
}
constexpr size_t kMaxSmemBytes = 227 * 1024;

template <typename T, int K, int R, typename CAPS = FullCaps, int ROWS = stash_rows<T>()>
struct RevCfg {
    using Caps = CAPS;
    static constexpr int NT = 1 << (K - R), NW = NT / 32;
    static constexpr RevOffsets ro =
        rev_offsets(K, R, FT<T>::L, FT<T>::AB, sizeof(T), Prog<T, R>::template Layout<CAPS>::bytes, ROWS);
    static constexpr size_t o_row = ro.row, o_prog = ro.prog, o_acc = ro.acc, o_stash = ro.stash, o_map = ro.map;
    static constexpr size_t smem() { return ro.bytes; }
    static_assert(ro.bytes <= kMaxSmemBytes, "reverse pass exceeds shared memory");
    static_assert(o_stash % 16 == 0, "stash rows are read with 16-byte loads");
};

template <typename T, int K, int R>
__global__ void __launch_bounds__(1 << (K - R))
    k_fused_rev(const amp_t<T> *__restrict__ phi_src, amp_t<T> *__restrict__ phi_dst,
                amp_t<T> *__restrict__ lam, const FPass *__restrict__ passes, int pi,
                const FStage *__restrict__ stages, const FOp *__restrict__ ops,
                const FDiag *__restrict__ diags, const FDItem *__restrict__ items,
                const int *__restrict__ slot_map, const typename FT<T>::mat_t *__restrict__ mats, uint64_t n_tiles,
                double *__restrict__ partials, int nb, int wmask) {
    using A = amp_t<T>;
    using C = RevCfg<T, K, R>;
    constexpr int NT = C::NT, NW = C::NW;
    extern __shared__ __align__(16) unsigned char smem[];
    A *tphi = reinterpret_cast<A *>(smem);
    A *tlam = tphi + (1 << K);
    uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + C::o_row);
    Prog<T, R> pg;
    pg.template bind<typename C::Caps>(smem + C::o_prog);
    double *acc = reinterpret_cast<double *>(smem + C::o_acc);
    T *stash = reinterpret_cast<T *>(smem + C::o_stash);
    int *smap = reinterpret_cast<int *>(smem + C::o_map);
    const FPass &P = passes[pi];
    const int tid = threadIdx.x;
    const int n_ls = P.n_lslots;
    fill_row_offsets<T, K>(P.high, row_off, tid, NT);
    for (int i = tid; i < n_ls; i += NT) acc[i] = 0.0, smap[i] = slot_map[P.slotmap0 + i];
    load_prog<T, R>(pg, P.rstage0, P.n_rstage, P.rdiag0, P.n_rdiag, stages, ops, diags, items, mats, true, tid, NT);
    __syncthreads();
    for (uint64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        if (ti + gridDim.x < n_tiles) {
            const uint64_t next = tile_base(ti + gridDim.x, P.nontile, P.n_nontile);
            TileIO<T, K>::template prefetch<NT>(phi_src, next, row_off, tid);
            TileIO<T, K>::template prefetch<NT>(lam, next, row_off, tid);
        }
        rev_tile<T, K, R, false>(tphi, tlam, row_off, pg, P.n_rstage, tile_base(ti, P.nontile, P.n_nontile),
                                 phi_src, phi_dst, lam, acc, stash, tid, (wmask & 1) != 0, (wmask & 2) != 0);
    }
    __syncthreads();
    for (int i = tid; i < n_ls; i += NT) partials[(size_t)smap[i] * nb + blockIdx.x] = acc[i];
    (void)NW;
}

// ------------------------------------------------------------------ Hamiltonian pass
// Per tile, each thread owns CPT 16-byte chunks of amplitudes and treats them in
// batches of 8 amplitudes held in registers.  For a term z of a group with flip mask x,
// the sign at global index j = base | tile bits is
//   (-1)^{popcount(j & z)} = (-1)^{popcount(base & z_nt)} (-1)^{popcount(t & z_l)},
// so the first factor is folded into the weight once per tile and the inner loop is a
// 32-bit popcount per amplitude.
// Groups of up to this many terms add each term into the batch factors directly; larger
// ones sum per class and transform (see ham_tile).
constexpr int kHamDirectTerms = 6;

template <typename T, int K>
struct HamCfg {
    static constexpr int NT = 256;
    static constexpr size_t o_row = (size_t)(1 << K) * FT<T>::AB;
    static constexpr size_t o_tab = o_row + sizeof(uint64_t) * (1 << (K - FT<T>::L));
    static constexpr size_t tab_bytes = (sizeof(uint32_t) * 6 + 2 * sizeof(T)) * kMaxHamGroups +
                                        (2 * sizeof(uint32_t) + sizeof(uint64_t) + 2 * 2 * sizeof(T)) * kMaxHamTerms;
    static constexpr size_t smem() { return o_tab + tab_bytes; }
};

// Shared-memory tables of one Hamiltonian pass.  Per term: the non-tile part of z (for
// the per-tile sign), the tile-local part z_l, the weight, and its "class": the bits of
// z_l at the positions where the amplitudes of one register batch differ (see
// ham_tile), with the matching sign pattern over the batch.
template <typename T, int K>
struct HamTab {
    static constexpr int AB = FT<T>::AB;
    uint64_t *t_znt;
    amp_t<T> *t_w, *t_weff;
    uint32_t *t_zl, *g_xs, *g_t0, *g_nt;
    // the terms of a group are sorted by class once per launch; g_cend[8 g + c] is the end
    // of class c's run, counted from the group's first term
    uint16_t *g_cend;
    // a single-term group's term, indexed by the group (no dependent second lookup);
    // g_w is its weight with the tile's sign, refreshed per tile.  g_kind says whether the
    // group's weights are all real (0), all imaginary (1) or mixed (2): a Pauli string's
    // weight is its real coefficient times i^{popcount(x & z)}, so it is real or imaginary
    uint32_t *g_zl, *g_cls, *g_kind;
    amp_t<T> *g_w;
    int ng, n_terms;
    VQG_DEV void bind(unsigned char *p) {
        t_znt = reinterpret_cast<uint64_t *>(p);
        t_w = reinterpret_cast<amp_t<T> *>(t_znt + kMaxHamTerms);
        t_weff = t_w + kMaxHamTerms;
        t_zl = reinterpret_cast<uint32_t *>(t_weff + kMaxHamTerms);
        g_cend = reinterpret_cast<uint16_t *>(t_zl + kMaxHamTerms);
        static_assert(8 * kMaxHamGroups * sizeof(uint16_t) == kMaxHamTerms * sizeof(uint32_t),
                      "class ends take the place of a per-term word");
        g_xs = reinterpret_cast<uint32_t *>(g_cend + 8 * kMaxHamGroups);
        g_t0 = g_xs + kMaxHamGroups;
        g_nt = g_t0 + kMaxHamGroups;
        g_zl = g_nt + kMaxHamGroups;
        g_cls = g_zl + kMaxHamGroups;
        g_w = reinterpret_cast<amp_t<T> *>(g_cls + kMaxHamGroups);  // 16-byte aligned: see tab_bytes
        g_kind = reinterpret_cast<uint32_t *>(g_w + kMaxHamGroups);
    }
    // class bit d = bit of z_l at the d-th varying position of a batch
    template <int D, int SH, int E0>
    static VQG_DEV uint32_t class_of(uint32_t zl) {
        uint32_t cls = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int pos = (E0 && d == 0) ? 0 : SH + d - E0;
            cls |= ((zl >> pos) & 1u) << d;
        }
        return cls;
    }
    // SORT: sort the terms of each multi-term group by class (the interpreted pass); the
    // specialised passes take the terms in plan order.
    template <int D, int SH, int E0, bool SORT = true>
    VQG_DEV void load(const HPass &P, const HGroup *__restrict__ groups, const HTerm *__restrict__ terms,
                      int tid, int nt) {
        ng = P.n_group;
        const int term_base = ng ? groups[P.group0].term0 : 0;
        n_terms = ng ? groups[P.group0 + ng - 1].term0 + groups[P.group0 + ng - 1].n_term - term_base : 0;
        for (int g = tid; g < ng; g += nt) {
            const HGroup G = groups[P.group0 + g];
            g_xs[g] = swz<AB>(G.xl);  // swz is linear: swz(t ^ x) = swz(t) ^ swz(x)
            g_t0[g] = (uint32_t)(G.term0 - term_base);
            g_nt[g] = (uint32_t)G.n_term;
            bool re = true, im = true;
            for (int i = 0; i < G.n_term; ++i) {
                re = re && terms[G.term0 + i].wi == 0.0;
                im = im && terms[G.term0 + i].wr == 0.0;
            }
            g_kind[g] = re ? 0u : (im ? 1u : 2u);
            if (G.n_term == 1) {
                const HTerm &tm = terms[G.term0];
                g_zl[g] = tm.zl;
                g_cls[g] = class_of<D, SH, E0>(tm.zl);
            }
        }
        for (int k = tid; k < n_terms; k += nt) {
            const HTerm tm = terms[term_base + k];
            t_znt[k] = tm.znt;
            // the term's class rides in bits 24..26 (z_l itself has at most 13 bits)
            t_zl[k] = tm.zl | (class_of<D, SH, E0>(tm.zl) << 24);
            if constexpr (sizeof(T) == 4) t_w[k] = mk<T>(tm.fr, tm.fi);
            else t_w[k] = mk<T>(tm.wr, tm.wi);
        }
        if constexpr (!SORT) return;
        __syncthreads();
        // one thread per multi-term group: insertion sort of its terms by class (stable),
        // then the class ends
        for (int g = tid; g < ng; g += nt) {
            const int j0 = (int)g_t0[g], m = (int)g_nt[g];
            if (m < 2) continue;
            for (int a = j0 + 1; a < j0 + m; ++a) {
                const uint64_t znt = t_znt[a];
                const uint32_t zl = t_zl[a];
                const amp_t<T> w = t_w[a];
                const uint32_t c = class_of<D, SH, E0>(zl);
                int b = a;
                while (b > j0 && class_of<D, SH, E0>(t_zl[b - 1]) > c) {
                    t_znt[b] = t_znt[b - 1];
                    t_zl[b] = t_zl[b - 1];
                    t_w[b] = t_w[b - 1];
                    --b;
                }
                t_znt[b] = znt;
                t_zl[b] = zl;
                t_w[b] = w;
            }
            int j = j0;
            for (uint32_t c = 0; c < 8; ++c) {
                while (j < j0 + m && class_of<D, SH, E0>(t_zl[j]) == c) ++j;
                g_cend[8 * g + c] = (uint16_t)(j - j0);
            }
        }
    }
};

// Batch geometry of the Hamiltonian pass: each thread owns CPT 16-byte chunks per tile
// (chunk c = tid + 256 m) and treats BCH of them (BA amplitudes) at a time.  Inside a
// batch the tile-local indices are t = t0 ^ delta with delta spanning D bits: bit 0 (the
// second amplitude of a complex64 chunk, E0 = 1) and the low bits of m above position
// SH.  Hence parity(t & z_l) = parity(t0 & z_l) ^ parity(d & cls(z_l)), d = the batch
// index, and a group's f over the batch is an 8-point Walsh-Hadamard transform of its
// terms' signed weights accumulated per class.
template <typename T, int K>
struct HamGeo {
    using IO = TileIO<T, K>;
    static constexpr int NT = 256;
    static constexpr int CPT = IO::CHUNKS / NT;
    static constexpr int BCH = CPT < 8 / IO::CA ? CPT : 8 / IO::CA;
    static constexpr int BA = BCH * IO::CA;
    static constexpr int D = BA == 8 ? 3 : (BA == 4 ? 2 : (BA == 2 ? 1 : 0));
    static constexpr int E0 = IO::CA == 2 ? 1 : 0;
    static constexpr int LOG_NT_ROWS = 5;  // log2(NT / CPR), CPR = 8 chunks per row
    static constexpr int SH = FT<T>::L + LOG_NT_ROWS;
};

// One tile of a Hamiltonian pass; returns this thread's partial of Re<psi|dlam>.
template <typename T, int K, bool L2ONLY>
VQG_DEV T ham_tile(amp_t<T> *tile, const uint64_t *row_off, HamTab<T, K> &tb, uint64_t base, bool first,
                   const amp_t<T> *__restrict__ psi, amp_t<T> *__restrict__ lam, int tid) {
    using A = amp_t<T>;
    using IO = TileIO<T, K>;
    using G = HamGeo<T, K>;
    constexpr int AB = FT<T>::AB, L = FT<T>::L, NT = 256;
    constexpr int CPT = G::CPT, BCH = G::BCH, BA = G::BA;
    static_assert(CPT % BCH == 0 && (1 << G::D) == BA, "batching");
    IO::template load<NT, L2ONLY>(tile, psi, base, row_off, tid);
    for (int k = tid; k < tb.n_terms; k += NT) {
        const A w = tb.t_w[k];
        tb.t_weff[k] = (__popcll(base & tb.t_znt[k]) & 1) ? mk<T>(-w.x, -w.y) : w;
    }
    for (int g = tid; g < tb.ng; g += NT)
        if (tb.g_nt[g] == 1) {
            const int j = (int)tb.g_t0[g];
            const A w = tb.t_w[j];
            tb.g_w[g] = (__popcll(base & tb.t_znt[j]) & 1) ? mk<T>(-w.x, -w.y) : w;
        }
    __syncthreads();
    T run = 0;
#pragma unroll 1
    for (int b0 = 0; b0 < CPT; b0 += BCH) {
        uint32_t t0, sw[BA];
        uint64_t gch[BCH];
        A mine[BA], out[BA], delta[BA];  // delta: this pass's contribution to lambda
#pragma unroll
        for (int i = 0; i < BCH; ++i) {
            const int c = tid + NT * (b0 + i);
            const int row = c / IO::CPR, col = c % IO::CPR;
            const uint32_t tc = (uint32_t)(row << L) | (uint32_t)(col * IO::CA);
            if (i == 0) t0 = tc;
            gch[i] = base | row_off[row] | (uint64_t)(col * IO::CA);
#pragma unroll
            for (int e = 0; e < IO::CA; ++e) {
                sw[i * IO::CA + e] = swz<AB>(tc + e);
                mine[i * IO::CA + e] = tile[sw[i * IO::CA + e]];
                out[i * IO::CA + e] = mk<T>((T)0, (T)0);
                delta[i * IO::CA + e] = mk<T>((T)0, (T)0);
            }
            // lambda so far goes straight into the output registers: its first use is the
            // final add, so the load's latency hides behind the group loop
            if (!first) {
                const float4 *g = reinterpret_cast<const float4 *>(lam + gch[i]);
                IO::unpack(L2ONLY ? __ldcg(g) : __ldcs(g), out + i * IO::CA);
            }
        }
        for (int g = 0; g < tb.ng; ++g) {
            const uint32_t xs = tb.g_xs[g];
            const int j0 = tb.g_t0[g], nt_g = tb.g_nt[g];
            if (nt_g == 0) continue;  // the diagonal group exists even without terms
            if (nt_g == 1 && tb.g_kind[g] < 2) {
                // one term with a real (or imaginary) weight w: the factor at batch amplitude
                // k is +-w, the sign bit parity(t0 & z_l) ^ parity(k & class) set straight
                // into w's sign (one logic op), then a real (or i times real) multiply-add
                const uint32_t zl = tb.g_zl[g], cls = tb.g_cls[g];
                const uint32_t s0 = (uint32_t)__popc(t0 & zl) << 31;
                const uint32_t c0 = cls << 31, c1 = (cls >> 1) << 31, c2 = (cls >> 2) << 31;
                const A w = tb.g_w[g];
                if (tb.g_kind[g] == 0) {
#pragma unroll
                    for (int k = 0; k < BA; ++k) {
                        const uint32_t sk = s0 ^ ((k & 1) ? c0 : 0u) ^ ((k & 2) ? c1 : 0u) ^ ((k & 4) ? c2 : 0u);
                        const T ws = flip_sign<T>(w.x, sk);
                        const A p = tile[sw[k] ^ xs];
                        delta[k].x = fma_t<T>(ws, p.x, delta[k].x);
                        delta[k].y = fma_t<T>(ws, p.y, delta[k].y);
                    }
                } else {  // w = i v: w p = (-v p.y, v p.x)
#pragma unroll
                    for (int k = 0; k < BA; ++k) {
                        const uint32_t sk = s0 ^ ((k & 1) ? c0 : 0u) ^ ((k & 2) ? c1 : 0u) ^ ((k & 4) ? c2 : 0u);
                        const T vs = flip_sign<T>(w.y, sk);
                        const A p = tile[sw[k] ^ xs];
                        delta[k].x = fma_t<T>(-vs, p.y, delta[k].x);
                        delta[k].y = fma_t<T>(vs, p.x, delta[k].y);
                    }
                }
                continue;
            }
            if (nt_g > 1) {
                // several terms: the factor at batch amplitude k is
                //   f(k) = sum_j w_j (-1)^{parity(t0 & z_j)} (-1)^{parity(k & class_j)}.
                // Small groups add each term's signed weight into the BA factors directly (a
                // logic op sets the sign); large ones sum the signed weights per class (the
                // terms are sorted by class, so each class is one run) and take the BA-point
                // Walsh-Hadamard transform.  KIND 0 / 1: every weight real / imaginary, so
                // only that component is summed and multiplied.
                auto multi = [&](auto kc, auto dc) {
                    constexpr int KIND = decltype(kc)::value;
                    constexpr bool DIRECT = decltype(dc)::value;
                    T ux[BA], uy[BA];
                    if constexpr (DIRECT) {
#pragma unroll
                        for (int k = 0; k < BA; ++k) ux[k] = (T)0, uy[k] = (T)0;
                        for (int j = j0; j < j0 + nt_g; ++j) {
                            const A w = tb.t_weff[j];
                            const uint32_t zl = tb.t_zl[j];
                            const uint32_t s0 = (uint32_t)__popc(t0 & zl) << 31;
                            const uint32_t c0 = (zl >> 24) << 31, c1 = (zl >> 25) << 31, c2 = (zl >> 26) << 31;
#pragma unroll
                            for (int k = 0; k < BA; ++k) {
                                const uint32_t sk =
                                    s0 ^ ((k & 1) ? c0 : 0u) ^ ((k & 2) ? c1 : 0u) ^ ((k & 4) ? c2 : 0u);
                                if constexpr (KIND != 1) ux[k] += flip_sign<T>(w.x, sk);
                                if constexpr (KIND != 0) uy[k] += flip_sign<T>(w.y, sk);
                            }
                        }
                    } else {
                        const uint16_t *ce = tb.g_cend + 8 * g;
                        int jb = j0;
#pragma unroll
                        for (int c = 0; c < BA; ++c) {
                            const int je = j0 + (int)ce[c];
                            T sx = (T)0, sy = (T)0;
                            for (int j = jb; j < je; ++j) {
                                const A w = tb.t_weff[j];
                                const uint32_t sj = (uint32_t)__popc(t0 & tb.t_zl[j]) << 31;
                                if constexpr (KIND != 1) sx += flip_sign<T>(w.x, sj);
                                if constexpr (KIND != 0) sy += flip_sign<T>(w.y, sj);
                            }
                            ux[c] = sx;
                            uy[c] = sy;
                            jb = je;
                        }
#pragma unroll
                        for (int h = 1; h < BA; h <<= 1)
#pragma unroll
                            for (int c = 0; c < BA; ++c)
                                if (!(c & h)) {
                                    if constexpr (KIND != 1) {
                                        const T a = ux[c], b = ux[c | h];
                                        ux[c] = a + b;
                                        ux[c | h] = a - b;
                                    }
                                    if constexpr (KIND != 0) {
                                        const T a = uy[c], b = uy[c | h];
                                        uy[c] = a + b;
                                        uy[c | h] = a - b;
                                    }
                                }
                    }
#pragma unroll
                    for (int k = 0; k < BA; ++k) {
                        const A p = tile[sw[k] ^ xs];
                        if constexpr (KIND == 0) {
                            delta[k].x = fma_t<T>(ux[k], p.x, delta[k].x);
                            delta[k].y = fma_t<T>(ux[k], p.y, delta[k].y);
                        } else if constexpr (KIND == 1) {
                            delta[k].x = fma_t<T>(-uy[k], p.y, delta[k].x);
                            delta[k].y = fma_t<T>(uy[k], p.x, delta[k].y);
                        } else {
                            delta[k] = cfma<T>(mk<T>(ux[k], uy[k]), p, delta[k]);
                        }
                    }
                };
                using I0 = std::integral_constant<int, 0>;
                using I1 = std::integral_constant<int, 1>;
                using I2 = std::integral_constant<int, 2>;
                using DT = std::true_type;
                using DF = std::false_type;
                const uint32_t kind = tb.g_kind[g];
                if (nt_g <= kHamDirectTerms) {
                    if (kind == 0) multi(I0{}, DT{});
                    else if (kind == 1) multi(I1{}, DT{});
                    else multi(I2{}, DT{});
                } else {
                    if (kind == 0) multi(I0{}, DF{});
                    else if (kind == 1) multi(I1{}, DF{});
                    else multi(I2{}, DF{});
                }
                continue;
            }
            // one term with a complex weight: f = +-w with the sign pattern of its class
            A f[BA];
            {
                const uint32_t zl = tb.g_zl[g], cls = tb.g_cls[g];
                const A w = tb.g_w[g];
                uint32_t m = (__popc(t0 & zl) & 1) ? 0xFFu : 0u;
                if (cls & 1u) m ^= 0xAAu;
                if (cls & 2u) m ^= 0xCCu;
                if (cls & 4u) m ^= 0xF0u;
#pragma unroll
                for (int k = 0; k < BA; ++k) f[k] = ((m >> k) & 1u) ? mk<T>(-w.x, -w.y) : w;
            }
#pragma unroll
            for (int k = 0; k < BA; ++k) delta[k] = cfma<T>(f[k], tile[sw[k] ^ xs], delta[k]);
        }
        // energy part of this pass: Re <psi|delta>, once per amplitude instead of per group
#pragma unroll
        for (int k = 0; k < BA; ++k) {
            run += mine[k].x * delta[k].x + mine[k].y * delta[k].y;
            out[k] = cadd<T>(out[k], delta[k]);
        }
#pragma unroll
        for (int i = 0; i < BCH; ++i) __stcs(reinterpret_cast<float4 *>(lam + gch[i]), IO::pack(out + i * IO::CA));
    }
    __syncthreads();
    return run;
}

// complex64: two 256-thread blocks per SM (shared memory allows two); complex128 arithmetic
// needs more registers than two blocks' share and gets them.
template <typename T, int K>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    k_fused_ham(const amp_t<T> *__restrict__ psi, amp_t<T> *__restrict__ lam,
                const HPass *__restrict__ hp, int pi, const HGroup *__restrict__ groups,
                const HTerm *__restrict__ terms, uint64_t n_tiles, double *__restrict__ partials, int nb) {
    using A = amp_t<T>;
    using C = HamCfg<T, K>;
    constexpr int NT = 256;
    extern __shared__ __align__(16) unsigned char smem[];
    A *tile = reinterpret_cast<A *>(smem);
    uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + C::o_row);
    HamTab<T, K> tb;
    tb.bind(smem + C::o_tab);
    __shared__ double wsum[NT / 32];
    const HPass &P = hp[pi];
    const int tid = threadIdx.x;
    fill_row_offsets<T, K>(P.high, row_off, tid, NT);
    using G = HamGeo<T, K>;
    tb.template load<G::D, G::SH, G::E0>(P, groups, terms, tid, NT);
    double eacc = 0.0;
    __syncthreads();
    for (uint64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        if (ti + gridDim.x < n_tiles) {
            const uint64_t next = tile_base(ti + gridDim.x, P.nontile, P.n_nontile);
            TileIO<T, K>::template prefetch<NT>(psi, next, row_off, tid);
            if (!P.first) TileIO<T, K>::template prefetch<NT>(lam, next, row_off, tid);
        }
        const T run = ham_tile<T, K, false>(tile, row_off, tb, tile_base(ti, P.nontile, P.n_nontile),
                                            P.first != 0, psi, lam, tid);
        eacc += (double)warp_tree<T>(run);
    }
    if ((tid & 31) == 0) wsum[tid >> 5] = eacc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += wsum[w];
        partials[(size_t)P.eslot * nb + blockIdx.x] = s;
    }
}


// ------------------------------------------------------------------ specialised passes
// Kernels generated for one pass of one plan (spec.cu) run these bodies: the same launch
// geometry, shared-memory program and tile I/O as k_fused_fwd / k_fused_rev, with the
// pass's stage and op sequence written out as straight-line code in Body::tile (every op
// type, register bit, stash row and block index a literal), so the op loop's dispatch,
// the register-bit switch and the register moves at its merge points disappear.
template <typename T, int K, int R, typename Body>
VQG_DEV void fwd_pass_spec(const amp_t<T> *__restrict__ src, amp_t<T> *__restrict__ dst,
                           const FPass *__restrict__ passes, int pi, const FStage *__restrict__ stages,
                           const FOp *__restrict__ ops, const FDiag *__restrict__ diags,
                           const FDItem *__restrict__ items, const typename FT<T>::mat_t *__restrict__ mats,
                           uint64_t n_tiles) {
    using C = FwdCfg<T, K, R>;
    constexpr int NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem[];
    amp_t<T> *tile = reinterpret_cast<amp_t<T> *>(smem);
    uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + C::o_row);
    Prog<T, R> pg;
    pg.template bind<typename C::Caps>(smem + C::o_prog);
    const FPass &P = passes[pi];
    const int tid = threadIdx.x;
    fill_row_offsets<T, K>(P.high, row_off, tid, NT);
    load_prog<T, R>(pg, P.stage0, P.n_stage, P.diag0, P.n_diag, stages, ops, diags, items, mats, false, tid, NT);
    __syncthreads();
    const uint64_t n_act = 1ull << P.n_active;  // later tiles hold zeros only (FPass::n_active)
    for (uint64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        if (ti >= n_act) {
            TileIO<T, K>::template store_zero<NT>(dst, tile_base(ti, P.nontile, P.n_nontile), row_off, tid);
            continue;
        }
        if (ti + gridDim.x < n_act && !P.from_zero)
            TileIO<T, K>::template prefetch<NT>(src, tile_base(ti + gridDim.x, P.nontile, P.n_nontile), row_off, tid,
                                                P.zero_in);
        Body::tile(tile, row_off, pg, tile_base(ti, P.nontile, P.n_nontile), P.from_zero != 0, src, dst, tid,
                   P.zero_in);
    }
}

template <typename T, int K, int R, typename Body, typename CAPS = FullCaps, int ROWS = stash_rows<T>()>
VQG_DEV void rev_pass_spec(const amp_t<T> *__restrict__ phi_src, amp_t<T> *__restrict__ phi_dst,
                           amp_t<T> *__restrict__ lam, const FPass *__restrict__ passes, int pi,
                           const FStage *__restrict__ stages, const FOp *__restrict__ ops,
                           const FDiag *__restrict__ diags, const FDItem *__restrict__ items,
                           const int *__restrict__ slot_map, const typename FT<T>::mat_t *__restrict__ mats,
                           uint64_t n_tiles, double *__restrict__ partials, int nb, int wmask) {
    using C = RevCfg<T, K, R, CAPS, ROWS>;
    constexpr int NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem[];
    amp_t<T> *tphi = reinterpret_cast<amp_t<T> *>(smem);
    amp_t<T> *tlam = tphi + (1 << K);
    uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + C::o_row);
    Prog<T, R> pg;
    pg.template bind<typename C::Caps>(smem + C::o_prog);
    double *acc = reinterpret_cast<double *>(smem + C::o_acc);
    T *stash = reinterpret_cast<T *>(smem + C::o_stash);
    int *smap = reinterpret_cast<int *>(smem + C::o_map);
    const FPass &P = passes[pi];
    const int tid = threadIdx.x;
    const int n_ls = P.n_lslots;
    fill_row_offsets<T, K>(P.high, row_off, tid, NT);
    for (int i = tid; i < n_ls; i += NT) acc[i] = 0.0, smap[i] = slot_map[P.slotmap0 + i];
    load_prog<T, R>(pg, P.rstage0, P.n_rstage, P.rdiag0, P.n_rdiag, stages, ops, diags, items, mats, true, tid, NT);
    __syncthreads();
    for (uint64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        if (ti + gridDim.x < n_tiles) {
            const uint64_t next = tile_base(ti + gridDim.x, P.nontile, P.n_nontile);
            TileIO<T, K>::template prefetch<NT>(phi_src, next, row_off, tid);
            TileIO<T, K>::template prefetch<NT>(lam, next, row_off, tid);
        }
        Body::tile(tphi, tlam, row_off, pg, tile_base(ti, P.nontile, P.n_nontile), phi_src, phi_dst, lam, acc,
                   stash, tid, (wmask & 1) != 0, (wmask & 2) != 0);
    }
    __syncthreads();
    for (int i = tid; i < n_ls; i += NT) partials[(size_t)smap[i] * nb + blockIdx.x] = acc[i];
}

template <typename T, int K, int R>
VQG_DEV void fwd_gather(const StageGeo<T, K, R> &g, const amp_t<T> *tile, amp_t<T> (&a)[1 << R]) {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) a[j] = tile[reg_addr<R, 1 << R>(g.sb, g.w, j)];
}
template <typename T, int K, int R>
VQG_DEV void fwd_scatter(StageGeo<T, K, R> &g, bool has_phase, amp_t<T> *tile, const amp_t<T> (&a)[1 << R],
                         amp_t<T> phase, T kacc) {
    constexpr int NA = 1 << R;
    asm volatile("" : "+r"(g.sb));  // recompute the addresses instead of keeping them live
    if (has_phase) {
        if constexpr (std::is_same<T, float>::value) phase = mk<T>(phase.x * kacc, phase.y * kacc);
#pragma unroll
        for (int j = 0; j < NA; ++j) tile[reg_addr<R, NA>(g.sb, g.w, j)] = cmul<T>(phase, a[j]);
    } else if (scaled_stage<T>(kacc)) {
        if constexpr (std::is_same<T, float>::value) {
            const float2 sv = make_float2(kacc, kacc);
#pragma unroll
            for (int j = 0; j < NA; ++j) tile[reg_addr<R, NA>(g.sb, g.w, j)] = __fmul2_rn(sv, a[j]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NA; ++j) tile[reg_addr<R, NA>(g.sb, g.w, j)] = a[j];
    }
}

// First and last stage of a specialised pass: they read the state from HBM into registers
// and write it back from registers, without the shared tile (one round trip through shared
// memory less per tile and state).  Amplitude j of the thread is global index gb | gm[j],
// gm[j] the global bits of the register bits set in j (literals of the generated code); the
// arithmetic on the way out is rev_scatter's / fwd_scatter's.
template <int R>
VQG_DEV void rev_gather_global(uint64_t gb, const uint64_t (&gm)[1 << R], const float2 *__restrict__ phi,
                               const float2 *__restrict__ lam, float2 (&a)[1 << R], float2 (&l)[1 << R]) {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        a[j] = __ldcs(phi + (gb | gm[j]));
        l[j] = __ldcs(lam + (gb | gm[j]));
    }
}
template <int R>
VQG_DEV void rev_scatter_global(uint64_t gb, const uint64_t (&gm)[1 << R], bool has_phase, float2 *__restrict__ phi,
                                float2 *__restrict__ lam, bool write_phi, bool write_lam, const float2 (&a)[1 << R],
                                const float2 (&l)[1 << R], float2 phase, float kacc) {
    constexpr int NA = 1 << R;
    asm volatile("" : "+l"(gb));  // form the addresses here instead of keeping them live
    const bool scaled = scaled_stage<float>(kacc);
    phase = make_float2(phase.x * kacc, phase.y * kacc);
    const float2 pr = make_float2(phase.x, phase.x), pi2 = make_float2(-phase.y, phase.y), sv = make_float2(kacc, kacc);
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        float2 va = a[j], vl = l[j];
        if (has_phase) {
            va = __ffma2_rn(pr, a[j], __fmul2_rn(pi2, make_float2(a[j].y, a[j].x)));
            vl = __ffma2_rn(pr, l[j], __fmul2_rn(pi2, make_float2(l[j].y, l[j].x)));
        } else if (scaled) {
            va = __fmul2_rn(sv, a[j]);
            vl = __fmul2_rn(sv, l[j]);
        }
        if (write_phi) __stcs(phi + (gb | gm[j]), va);
        if (write_lam) __stcs(lam + (gb | gm[j]), vl);
    }
}
template <int R>
VQG_DEV void fwd_gather_global(uint64_t gb, const uint64_t (&gm)[1 << R], bool from_zero,
                               const float2 *__restrict__ src, float2 (&a)[1 << R], uint64_t zmask) {
    if (from_zero) {  // |0...0>
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) a[j] = make_float2((gb | gm[j]) == 0 ? 1.f : 0.f, 0.f);
    } else {  // amplitudes known zero (FPass::zero_in) are not read
#pragma unroll
        for (int j = 0; j < (1 << R); ++j)
            a[j] = ((gb | gm[j]) & zmask) ? make_float2(0.f, 0.f) : __ldcs(src + (gb | gm[j]));
    }
}
template <int R>
VQG_DEV void fwd_scatter_global(uint64_t gb, const uint64_t (&gm)[1 << R], bool has_phase, float2 *__restrict__ dst,
                                const float2 (&a)[1 << R], float2 phase, float kacc) {
    constexpr int NA = 1 << R;
    asm volatile("" : "+l"(gb));  // form the addresses here instead of keeping them live
    const bool scaled = scaled_stage<float>(kacc);
    phase = make_float2(phase.x * kacc, phase.y * kacc);
    const float2 sv = make_float2(kacc, kacc);
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        float2 v = a[j];
        if (has_phase) v = cmul<float>(phase, a[j]);
        else if (scaled) v = __fmul2_rn(sv, a[j]);
        __stcs(dst + (gb | gm[j]), v);
    }
}

// Reverse diagonal block, split for the specialised kernels (rev_diag does both parts for
// the interpreted pass, for any item list): rev_diag_sums forms the block's input sums
// H[k] = sum over register index bit k = 0 of p_j and S = sum of all p_j, with
// p_j = Im(conj(lambda_j) phi_j), from the same pairwise tree as rev_diag; an RZ on register
// bit k then has Im<lambda|Z|phi> = 2 H[k] - S, one on a thread-level qubit +-S.
template <int R>
VQG_DEV void rev_diag_sums(const float2 (&a)[1 << R], const float2 (&l)[1 << R], float (&H)[R], float &S) {
    constexpr int NA = 1 << R;
    float2 q[NA / 2];
#pragma unroll
    for (int m = 0; m < NA / 2; ++m)
        q[m] = make_float2(l[2 * m].x * a[2 * m].y - l[2 * m].y * a[2 * m].x,
                           l[2 * m + 1].x * a[2 * m + 1].y - l[2 * m + 1].y * a[2 * m + 1].x);
#pragma unroll
    for (int k = 1; k < R; ++k) {  // fold index bit k (bit k - 1 of m)
        const int len = (NA / 2) >> (k - 1);
        float2 h = q[0];
#pragma unroll
        for (int m = 1; m < len / 2; ++m) h = __fadd2_rn(h, q[2 * m]);
        H[k] = h.x + h.y;
#pragma unroll
        for (int m = 0; m < len / 2; ++m) q[m] = __fadd2_rn(q[2 * m], q[2 * m + 1]);
    }
    H[0] = q[0].x;
    S = q[0].x + q[0].y;
}
// d * a in four scalar FP32 operations (a packed form needs the swapped pair (a.y, a.x)
// built by moves and measured no faster).
VQG_DEV float2 cmul_scalar(float2 d, float2 a) {
    return make_float2(__fmaf_rn(-d.y, a.y, __fmul_rn(d.x, a.x)), __fmaf_rn(d.y, a.x, __fmul_rn(d.x, a.y)));
}

// The block's table on phi and lambda (rev_diag's second part); the per-thread factor tau
// and the sign mask c are computed by the generated code from the block's thread-level
// items (literal qubits) and the pending phase takes tau.  The sign pattern only exists
// where the block has a CZ between a register bit and a thread-level qubit (HAS_RT).
template <int R, bool HAS_RT>
VQG_DEV void rev_diag_table(float2 (&a)[1 << R], float2 (&l)[1 << R], const float2 *tab, uint32_t c) {
    constexpr int NA = 1 << R;
    uint32_t w = 0;
    if constexpr (HAS_RT) w = walsh_bits(c);
    const float4 *t4 = reinterpret_cast<const float4 *>(tab);  // two entries per 16-byte load
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const float4 q = t4[j >> 1];
        float2 dj = (j & 1) ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
        if constexpr (HAS_RT)
            if ((w >> j) & 1u) dj = neg<float>(dj);
        a[j] = cmul_scalar(dj, a[j]);
        l[j] = cmul_scalar(dj, l[j]);
    }
}

// Forward op bodies for the specialised kernels (the interpreted pass runs apply_fwd_op).
template <int KB, int R, typename T>
VQG_DEV void fwd_op_ry(amp_t<T> (&a)[1 << R], const amp_t<T> *m, T &kacc) {
    if constexpr (std::is_same<T, float>::value) {
        const float2 p1 = m[1];
        op_ry_scaled<KB, 1 << R>(a, p1.x, p1.y != 0.f);
        kacc *= m[2].x;
    } else {
        const amp_t<T> cs = m[0];
        op_ry<KB, 1 << R, T>(a, cs.x, cs.y);
    }
}
// The forward counterpart of rev_diag_table (psi only).
template <int R, bool HAS_RT>
VQG_DEV void fwd_diag_table(float2 (&a)[1 << R], const float2 *tab, uint32_t c) {
    constexpr int NA = 1 << R;
    uint32_t w = 0;
    if constexpr (HAS_RT) w = walsh_bits(c);
    const float4 *t4 = reinterpret_cast<const float4 *>(tab);
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const float4 q = t4[j >> 1];
        float2 dj = (j & 1) ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
        if constexpr (HAS_RT)
            if ((w >> j) & 1u) dj = neg<float>(dj);
        a[j] = cmul_scalar(dj, a[j]);
    }
}


// Specialised Hamiltonian pass (spec.cu), complex64: ham_tile with the group loop replaced
// by the generated Body::groups, which visits the pass's groups with their flip masks, term
// masks, classes and weight kinds as literals (weights and the tile's signs still come from
// the shared-memory table, in plan order).
//
// Amplitudes are held in slot order: a 16-byte chunk of the tile holds the two amplitudes
// t and t ^ 1 (swz(t ^ 1) = swz(t) ^ 1), in an order given by bit 0 of swz(t), which the
// swizzle folds from higher index bits (b_i, per chunk at run time).  Slot j of own chunk i
// (logical amplitude j ^ b_i) has its partner under a flip mask x at slot j ^ x0 of the chunk
// at B_i ^ (swz(x) & ~1): the partners of both slots come with one 16-byte load and their
// positions are literals (the generated body shares these loads between flip masks that
// differ only in the batch's own bits, and takes the batch's own chunks, mine, where a mask
// has no other bits).  b_i enters only the sign of terms whose class has bit 0 (b31[i] =
// b_i << 31), and the logical order is restored once per batch when lambda is written.
template <int K, bool L2ONLY, typename Body>
VQG_DEV float ham_tile_spec(float2 *tile, const uint64_t *row_off, HamTab<float, K> &tb, uint64_t base, bool first,
                            const float2 *__restrict__ psi, float2 *__restrict__ lam, int tid) {
    using A = float2;
    using IO = TileIO<float, K>;
    using G = HamGeo<float, K>;
    constexpr int AB = 8, L = FT<float>::L, NT = 256;
    constexpr int CPT = G::CPT, BCH = G::BCH, BA = G::BA;
    static_assert(IO::CA == 2 && BA == 2 * BCH, "two amplitudes per chunk");
    IO::template load<NT, L2ONLY>(tile, psi, base, row_off, tid);
    for (int k = tid; k < tb.n_terms; k += NT) {
        const A w = tb.t_w[k];
        tb.t_weff[k] = (__popcll(base & tb.t_znt[k]) & 1) ? mk<float>(-w.x, -w.y) : w;
    }
    for (int g = tid; g < tb.ng; g += NT)
        if (tb.g_nt[g] == 1) {
            const int j = (int)tb.g_t0[g];
            const A w = tb.t_w[j];
            tb.g_w[g] = (__popcll(base & tb.t_znt[j]) & 1) ? mk<float>(-w.x, -w.y) : w;
        }
    __syncthreads();
    float run = 0;
#pragma unroll 1
    for (int b0 = 0; b0 < CPT; b0 += BCH) {
        uint32_t t0, B[BCH], b31[BCH];
        uint64_t gch[BCH];
        A mine[BA], out[BA], delta[BA];  // mine, delta: slot order; out: logical order
#pragma unroll
        for (int i = 0; i < BCH; ++i) {
            const int c = tid + NT * (b0 + i);
            const int row = c / IO::CPR, col = c % IO::CPR;
            const uint32_t tc = (uint32_t)(row << L) | (uint32_t)(col * IO::CA);
            if (i == 0) t0 = tc;
            gch[i] = base | row_off[row] | (uint64_t)(col * IO::CA);
            const uint32_t sw = swz<AB>(tc);
            B[i] = sw & ~1u;
            b31[i] = sw << 31;
            const float4 m = *reinterpret_cast<const float4 *>(tile + B[i]);
            mine[2 * i] = make_float2(m.x, m.y);
            mine[2 * i + 1] = make_float2(m.z, m.w);
            out[2 * i] = out[2 * i + 1] = delta[2 * i] = delta[2 * i + 1] = make_float2(0.f, 0.f);
            if (!first) {
                const float4 *g = reinterpret_cast<const float4 *>(lam + gch[i]);
                IO::unpack(L2ONLY ? __ldcg(g) : __ldcs(g), out + 2 * i);
            }
        }
        Body::groups(tb, tile, t0, B, b31, mine, delta);
#pragma unroll
        for (int k = 0; k < BA; ++k) run += mine[k].x * delta[k].x + mine[k].y * delta[k].y;
#pragma unroll
        for (int i = 0; i < BCH; ++i) {
            const bool swp = b31[i] != 0u;  // logical amplitude e sits at slot e ^ b_i
            const A d0 = swp ? delta[2 * i + 1] : delta[2 * i], d1 = swp ? delta[2 * i] : delta[2 * i + 1];
            out[2 * i] = cadd<float>(out[2 * i], d0);
            out[2 * i + 1] = cadd<float>(out[2 * i + 1], d1);
            __stcs(reinterpret_cast<float4 *>(lam + gch[i]), IO::pack(out + 2 * i));
        }
    }
    __syncthreads();
    return run;
}

template <typename T, int K, typename Body>
VQG_DEV void ham_pass_spec(const amp_t<T> *__restrict__ psi, amp_t<T> *__restrict__ lam, const HPass *__restrict__ hp,
                           int pi, const HGroup *__restrict__ groups, const HTerm *__restrict__ terms, uint64_t n_tiles,
                           double *__restrict__ partials, int nb) {
    using C = HamCfg<T, K>;
    constexpr int NT = 256;
    extern __shared__ __align__(16) unsigned char smem[];
    amp_t<T> *tile = reinterpret_cast<amp_t<T> *>(smem);
    uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + C::o_row);
    HamTab<T, K> tb;
    tb.bind(smem + C::o_tab);
    __shared__ double wsum[NT / 32];
    const HPass &P = hp[pi];
    const int tid = threadIdx.x;
    fill_row_offsets<T, K>(P.high, row_off, tid, NT);
    using G = HamGeo<T, K>;
    tb.template load<G::D, G::SH, G::E0, false>(P, groups, terms, tid, NT);
    double eacc = 0.0;
    __syncthreads();
    for (uint64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        if (ti + gridDim.x < n_tiles) {
            const uint64_t next = tile_base(ti + gridDim.x, P.nontile, P.n_nontile);
            TileIO<T, K>::template prefetch<NT>(psi, next, row_off, tid);
            if (!P.first) TileIO<T, K>::template prefetch<NT>(lam, next, row_off, tid);
        }
        const T run = ham_tile_spec<K, false, Body>(tile, row_off, tb, tile_base(ti, P.nontile, P.n_nontile),
                                                    P.first != 0, psi, lam, tid);
        eacc += (double)warp_tree<T>(run);
    }
    if ((tid & 31) == 0) wsum[tid >> 5] = eacc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += wsum[w];
        partials[(size_t)P.eslot * nb + blockIdx.x] = s;
    }
}

}  // namespace vqg
