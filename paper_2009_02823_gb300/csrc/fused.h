// Plan records of the tile-fused sweeps, shared by the host planner (engine.cu) and
// the kernels (fused_kernels.cuh, instantiated in k_fused_c64.cu, k_fused_c128.cu,
// k_fused_ham.cu and batch.cu).
//
// A tile is 2^K amplitudes: the L lowest qubits (contiguous 128-byte rows of the
// state) plus K-L chosen "high" qubits; the other n-K qubits are fixed per tile.  One
// pass streams every tile through shared memory once and applies a run of gates
// whose non-diagonal qubits lie in the tile (diagonal gates and CNOT controls can
// sit anywhere: their index bits are known).  Inside a pass, stages gather 2^R
// amplitudes per thread into registers (R "register qubits"), apply every gate of
// the stage there, and scatter back.
#pragma once

#include <stdint.h>

namespace vqg {

constexpr int kMaxHigh = 24;
constexpr int kMaxNontile = 40;
constexpr int kMaxThreadBits = 12;
constexpr int kMaxRegBits = 5;
constexpr int kMaxPassOps = 192;     // register-stage ops (gates or diagonal blocks) per pass
constexpr int kMaxPassStages = 64;
constexpr int kMaxPassSlots = 256;   // reverse reduction values per pass
constexpr int kMaxPassDiags = 48;    // diagonal blocks per pass
constexpr int kMaxPassItems = 320;   // diagonal-block items per pass
constexpr int kMaxDiagRz = 8;        // RZ gates per diagonal block
constexpr int kMaxDiagCz = 16;       // CZ gates per diagonal block
constexpr int kMaxStageRows = 16;    // reverse reduction values per register stage (complex64)
constexpr int kMaxStageRowsDbl = 8;  // the same for complex128 (FP64 stash)
constexpr int kMaxStageValues = 64;  // reverse reduction values per register stage (stash flushed)
constexpr int kMaxHamGroups = 256;   // groups per Hamiltonian pass
constexpr int kMaxHamTerms = 1024;   // terms per Hamiltonian pass

// Per-pass program budget of a kernel's shared-memory program; the planner keeps every
// pass within the budget of the kernel that will run it.
struct PassCaps {
    int ops, stages, diags, items;
};
template <int OPS, int STAGES, int DIAGS, int ITEMS>
struct CapsT {
    static constexpr int ops = OPS, stages = STAGES, diags = DIAGS, items = ITEMS;
    static constexpr PassCaps value() { return {OPS, STAGES, DIAGS, ITEMS}; }
};
using FullCaps = CapsT<kMaxPassOps, kMaxPassStages, kMaxPassDiags, kMaxPassItems>;
// The batched launch's smaller program keeps two 256-thread blocks resident per SM.
using BatchCaps = CapsT<96, 32, 24, 160>;

enum FOpType : int16_t {
    OP_RY = 0,    // real rotation on register bit k
    OP_RX = 1,    // RX on register bit k (complex matrix)
    OP_U3 = 2,    // general 2x2 on register bit k (three parameters)
    OP_CNOT = 3,  // swap on target register bit k where the control is set
    OP_DIAG = 4,  // a block of commuting diagonal gates (RZ, CZ): table x per-thread factor
    // 2x2 matrix on target register bit k where the control is set (rm0: control register
    // mask; else cq: control qubit, -1 = no control); they differ in the reverse
    // reduction: Im<l|P X|phi>, Im<l|P Y|phi>, Im<l|P Z|phi>, -2 Im<l|P |1><1| phi>
    OP_CRX = 5,
    OP_CRY = 6,
    OP_CRZ = 7,
    OP_PH = 8,    // phase gate (uncontrolled: PHASE; controlled: CPHASE)
    // reverse only: reduce the stash rows written so far in this stage (row = count) into
    // local slots lslot .. lslot + row - 1, so that a stage can carry more reduction values
    // than the stash has rows without a new gather/scatter
    OP_FLUSH = 9,
    OP_LAST = OP_FLUSH
};

// Items of a diagonal block.  RZ items come first (they carry reverse reductions).
enum FDItemType : int16_t {
    DI_RZ_REG = 0,  // RZ on register bit k0 (in the block's table)
    DI_RZ_THR = 1,  // RZ on a thread- or tile-level qubit g0 (per-thread phase)
    DI_CZ_RR = 2,   // CZ on register bits k0, k1 (in the table)
    DI_CZ_RT = 3,   // CZ on register bit k0 and thread-level qubit g0 (per-thread sign mask)
    DI_CZ_TT = 4    // CZ on thread-level qubits g0, g1 (per-thread sign)
};

struct FPass {
    int32_t high[kMaxHigh];        // global qubit at tile position L + i
    int32_t nontile[kMaxNontile];  // global qubits outside the tile: the n_active that may hold
                                   // set bits first, then the rest (each part ascending)
    int32_t n_high, n_nontile;
    int32_t stage0, n_stage;       // forward stages
    int32_t rstage0, n_rstage;     // reverse stages
    int32_t n_lslots;              // reverse: reduction values accumulated by this pass
    int32_t slotmap0;              // reverse: first entry of this pass in the slot map
    int32_t from_zero;             // forward: the input is |0...0> (nothing to load)
    int32_t n_gates;               // gates applied by this pass
    int32_t diag0, n_diag;         // forward diagonal blocks
    int32_t rdiag0, n_rdiag;       // reverse diagonal blocks
    // Tiles whose index has a bit set at or above n_active hold only zero amplitudes: the
    // sweep starts from |0...0> and no gate before this pass moved amplitude onto those
    // non-tile qubits.  The forward pass writes zeros there without computing; the reverse
    // pass skips them (phi is zero there, so they add nothing to any gradient, and the
    // earlier passes never read their lambda).  n_active = n_nontile: every tile computed.
    int32_t n_active;
    int32_t n_active_zero;         // host: n_active for a |0...0> start (an input state: all)
    // Index bits on which the pass's input is zero (qubits outside the support before the
    // pass, for a |0...0> start; 0 with an input state): the forward pass reads an input
    // amplitude only where its index has none of these bits and takes zero elsewhere, so the
    // passes before it need not write the zeros of the tiles they skip.
    uint64_t zero_in;
    uint64_t zero_in_zero;         // host: zero_in for a |0...0> start
};

struct FStage {
    uint16_t thr_sw[kMaxThreadBits];     // swizzled tile-local mask of thread bit b
    uint16_t reg_sw[kMaxRegBits + 3];    // swizzled tile-local mask of register bit k
    int8_t thr_q[kMaxThreadBits];        // global qubit of thread bit b
    int32_t op0, n_op;
    int16_t row_slot[kMaxStageRows];     // reverse: local reduction slot of each stash row
    int16_t n_rows;                      // reverse: stash rows used by this stage
    int16_t has_phase;                   // a diagonal block of the stage has a per-thread phase
};

struct FOp {          // 16 bytes: one shared-memory vector load
    int8_t type, k;   // k: register bit of the non-diagonal target
    int8_t cq;        // CNOT: global qubit of a control that is not a register bit, else -1
    int8_t row;       // reverse: first stash row of this op's reduction values
    int16_t diag;     // OP_DIAG: block index within the pass
    int16_t lslot;    // reverse: first local reduction value (-1: none)
    uint32_t rm0;     // CNOT: register mask of the control (0: control not a register bit)
    int32_t gate;     // gate index (matrix source); OP_DIAG: -1
};

// Items of a block are ordered RZ on register bits, RZ on thread-level qubits, CZ with
// a thread-level qubit (CZ_RT, CZ_TT), CZ between register bits: the RZ items lead (they
// carry reverse reductions) and the per-thread factor only visits [thr0, thr0 + n_thr).
struct FDiag {
    int32_t item0, n_item;  // items (global index)
    int16_t n_rz;           // leading RZ items
    int16_t has_rt;         // any CZ between a register bit and a thread-level qubit
    int16_t thr0, n_thr;    // thread-level items, relative to item0
};

struct FDItem {
    int16_t type, k0, k1, pad;
    int32_t gate;   // RZ: gate index (phases)
    int32_t lslot;  // reverse RZ: local reduction slot
    uint64_t g0, g1;
};

// Hamiltonian tile pass: groups whose flip mask lies inside the tile.
struct HPass {
    int32_t high[kMaxHigh];
    int32_t nontile[kMaxNontile];
    int32_t n_high, n_nontile;
    int32_t group0, n_group;
    int32_t first;  // writes lambda (no accumulate)
    int32_t eslot;  // energy partial slot
};

struct HGroup {
    uint64_t xg;     // global flip mask
    uint32_t xl;     // tile-local flip mask
    int32_t term0, n_term;
    int32_t pad;
};

// Term of a group, evaluated at the source index j^x: w' = w * (-1)^{popcount(x & z)}.
struct HTerm {
    uint64_t z;     // global z mask
    uint64_t znt;   // the part of z on qubits outside the tile of its pass
    double wr, wi;
    float fr, fi;   // the same weight rounded to FP32 (complex64 kernels)
    uint32_t zl;    // the part of z inside the tile, as tile-local positions
    int32_t pad;
};

// Swizzle of a tile-local amplitude index into its shared-memory slot: XOR-folds the
// bits above the 128-byte row into the position within the row, so that 16 (8) lanes
// touching indices whose varying bits have distinct residues mod 4 (mod 3) hit
// distinct banks.  Linear over GF(2); keeps rows intact.
template <int AMP_BYTES>
__host__ __device__ constexpr uint32_t swz(uint32_t t) {
    if (AMP_BYTES == 8) return t ^ (((t >> 4) ^ (t >> 8) ^ (t >> 12) ^ (t >> 16)) & 15u);
    return t ^ (((t >> 3) ^ (t >> 6) ^ (t >> 9) ^ (t >> 12) ^ (t >> 15)) & 7u);
}

}  // namespace vqg
