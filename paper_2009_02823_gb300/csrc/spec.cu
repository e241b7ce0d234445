// Per-pass specialised kernels for the complex64 tile passes.
//
// The interpreted passes (k_fused_fwd, k_fused_rev) read each op's descriptor from shared
// memory, branch on its type and on its register bit, and merge the branches' register
// assignments after every op; that control work is most of their instruction stream.  A
// specialised kernel runs the same pass with its stage and op sequence written out as
// straight-line code: the op types, register bits, stash rows, diagonal-block indices and
// flush points become literals, while everything that depends on theta (rotation factors,
// diagonal tables, per-thread phases) is still read from the pass's shared-memory program
// exactly as the interpreter reads it.  Arithmetic, order of operations and reductions
// are the interpreter's, so results are identical.
//
// The source of each pass's kernel is generated here from the host plan, compiled by
// nvcc into a cubin (cached on disk by a hash of the source and the compiler command),
// loaded with cudaLibraryLoadData and launched with cudaLaunchKernel on the circuit's
// stream.  Compilation needs nvcc (VQG_NVCC, $CUDA_HOME/bin/nvcc, /usr/local/cuda/bin/nvcc
// or PATH) and the library's own headers, found next to libvqg.so (or in VQG_SPEC_SRC and
// VQG_SPEC_INC).  The cache directory is VQG_SPEC_CACHE (default $TMPDIR/vqg_spec_<uid>).
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"
#include "fused_kernels.cuh"
#include "plan.h"

namespace vqg {

namespace {

const char *kRevArgs =
    "const float2 *__restrict__ phi_src, float2 *__restrict__ phi_dst, float2 *__restrict__ lam, "
    "const vqg::FPass *__restrict__ passes, int pi, const vqg::FStage *__restrict__ stages, "
    "const vqg::FOp *__restrict__ ops, const vqg::FDiag *__restrict__ diags, const vqg::FDItem *__restrict__ items, "
    "const int *__restrict__ slot_map, const float *__restrict__ mats, uint64_t n_tiles, "
    "double *__restrict__ partials, int nb, int wmask";
const char *kRevNames = "phi_src, phi_dst, lam, passes, pi, stages, ops, diags, items, slot_map, mats, n_tiles, partials, nb, wmask";
const char *kFwdArgs =
    "const float2 *__restrict__ src, float2 *__restrict__ dst, const vqg::FPass *__restrict__ passes, int pi, "
    "const vqg::FStage *__restrict__ stages, const vqg::FOp *__restrict__ ops, const vqg::FDiag *__restrict__ diags, "
    "const vqg::FDItem *__restrict__ items, const float *__restrict__ mats, uint64_t n_tiles";
const char *kFwdNames = "src, dst, passes, pi, stages, ops, diags, items, mats, n_tiles";

// Thread-control expression of a controlled op (thread_control in the kernels).
std::string ctrl_expr(const FOp &op) {
    if (op.rm0) return "false";
    if (op.cq < 0) return "true";
    return "(((gb >> " + std::to_string((int)op.cq) + ") & 1ull) != 0)";
}

std::string prm(int o) { return "pg.prm + " + std::to_string(4 * o); }

// A stage reads and writes HBM directly only when no register bit is one of the row qubits
// 0..L-1: its lanes then run over those qubits (the thread bits take the lowest free tile
// positions of each residue mod 4 first), so a warp's access for one register index covers
// whole 128-byte rows.  Other stages go through the shared tile, whose loads and stores
// are row-coalesced by construction.
bool direct_io(const Plan &pl, int stage, int R) {
    for (int k = 0; k < R; ++k)
        if (pl.stage_reg_q[stage][k] < pl.L) return false;
    return true;
}

// Global-index offsets of a stage's register indices: gm[j] has the global bit of every
// register bit set in j (the first and last stage of a pass address HBM directly).
std::string gm_decl(const Plan &pl, int stage, int R) {
    std::ostringstream o;
    o << "const uint64_t gm[" << (1 << R) << "] = {";
    for (int j = 0; j < (1 << R); ++j) {
        uint64_t m = 0;
        for (int k = 0; k < R; ++k)
            if ((j >> k) & 1) m |= 1ull << pl.stage_reg_q[stage][k];
        o << (j ? ", " : "") << "0x" << std::hex << m << std::dec << "ull";
    }
    o << "};";
    return o.str();
}

// Literal per-thread factor of diagonal block D (what diag_thread computes from the item
// table at run time): tau from the RZ phases and CZ signs on thread-level qubits, folded
// into the stage's pending phase, and the sign mask c of the register-thread CZs.
std::string diag_thread_code(const Plan &pl, const FDiag &D, int item_base, const char *ind) {
    std::ostringstream o;
    bool tau = false, sign = false;
    o << ind << "uint32_t c = 0u; (void)c;\n";
    for (int k = D.thr0; k < D.thr0 + D.n_thr; ++k) {
        const FDItem &x = pl.items[D.item0 + k];
        const int rel = D.item0 + k - item_base;
        const int q0 = x.g0 ? __builtin_ctzll(x.g0) : 0, q1 = x.g1 ? __builtin_ctzll(x.g1) : 0;
        if (x.type == DI_RZ_THR) {
            const std::string f = "pg.iph[" + std::to_string(2 * rel) + " + (int)((gb >> " + std::to_string(q0) + ") & 1ull)]";
            if (!tau) o << ind << "A tau = " << f << ";\n";
            else o << ind << "tau = cmul<T>(" << f << ", tau);\n";
            tau = true;
        } else if (x.type == DI_CZ_TT) {
            if (!sign) o << ind << "uint32_t ng = 0u;\n";
            sign = true;
            o << ind << "ng ^= (uint32_t)((gb >> " << q0 << ") & (gb >> " << q1 << ") & 1ull);\n";
        } else if (x.type == DI_CZ_RT) {
            o << ind << "c ^= (uint32_t)((gb >> " << q0 << ") & 1ull) << " << (int)x.k0 << ";\n";
        }
    }
    if (sign) {
        if (!tau) o << ind << "A tau = mk<T>((T)1, (T)0);\n";
        o << ind << "if (ng) tau = neg<T>(tau);\n";
        tau = true;
    }
    if (tau) o << ind << "phase = cmul<T>(tau, phase);\n";
    return o.str();
}

// Straight-line body of one forward pass (mirrors fwd_tile + apply_fwd_op).
std::string gen_fwd(const Plan &pl, int pass) {
    const FPass &P = pl.passes[pass];
    const int K = pl.K, R = pl.Rf, NT = 1 << (K - R);
    const int op_base = P.n_stage ? pl.stages[P.stage0].op0 : 0;
    std::ostringstream o;
    o << "#include \"fused_kernels.cuh\"\n"
      << "namespace vqg { namespace spec {\n"
      << "struct Body {\n"
      << "  static VQG_DEV void tile(float2 *tile, const uint64_t *row_off, const Prog<float, " << R
      << "> &pg, uint64_t base, bool from_zero, const float2 *__restrict__ src, float2 *__restrict__ dst, int tid, "
         "uint64_t zin) {\n"
      << "    using T = float; using A = float2; using IO = TileIO<T, " << K << ">;\n"
      << "    constexpr int NT = " << NT << ", NA = " << (1 << R) << "; (void)NA;\n"
      << "    (void)row_off; (void)IO{};\n";
    const bool dfirst = P.n_stage > 0 && direct_io(pl, P.stage0, R);
    const bool dlast = P.n_stage > 0 && direct_io(pl, P.stage0 + P.n_stage - 1, R);
    if (!dfirst)
        o << "    if (from_zero) IO::template zero<NT>(tile, base, tid);\n"
          << "    else IO::template load<NT, false>(tile, src, base, row_off, tid, zin);\n"
          << "    __syncthreads();\n";
    for (int s = 0; s < P.n_stage; ++s) {
        const FStage &st = pl.stages[P.stage0 + s];
        const bool first = s == 0 && dfirst, last = s == P.n_stage - 1 && dlast;
        o << "    {  // stage " << s << "\n"
          << "      StageGeo<T, " << K << ", " << R << "> g; g.init(pg.st[" << s << "], tid, base);\n"
          << "      const uint64_t gb = g.gb; (void)gb;\n";
        if (first || last) o << "      " << gm_decl(pl, P.stage0 + s, R) << "\n";
        if (first) o << "      A a[NA]; fwd_gather_global<" << R << ">(gb, gm, from_zero, src, a, zin);\n";
        else o << "      A a[NA]; fwd_gather<T, " << K << ", " << R << ">(g, tile, a);\n";
        o << "      A phase = mk<T>((T)1, (T)0); T kacc = (T)1;\n";
        for (int i = 0; i < st.n_op; ++i) {
            const int oi = st.op0 + i, ol = oi - op_base;
            const FOp &op = pl.ops[oi];
            const std::string kb = std::to_string((int)op.k);
            switch (op.type) {
            case OP_RY:
                o << "      fwd_op_ry<" << kb << ", " << R << ", T>(a, " << prm(ol) << ", kacc);\n";
                break;
            case OP_RX:
            case OP_U3:
                o << "      op_gen<" << kb << ", NA, T>(a, mat_of<T>(" << prm(ol) << "));\n";
                break;
            case OP_CNOT:
                o << "      op_cnot<" << kb << ", NA, T>(a, " << op.rm0 << "u, "
                  << (op.rm0 ? std::string("false") : "(((gb >> " + std::to_string((int)op.cq) + ") & 1ull) != 0)")
                  << ");\n";
                break;
            case OP_CRX:
            case OP_CRY:
            case OP_CRZ:
            case OP_PH:
                o << "      op_cgen<" << kb << ", NA, T>(a, mat_of<T>(" << prm(ol) << "), " << op.rm0 << "u, "
                  << ctrl_expr(op) << ");\n";
                break;
            case OP_DIAG: {
                const FDiag &D = pl.diags[P.diag0 + op.diag];
                o << "      {  // diagonal block " << op.diag << "\n"
                  << diag_thread_code(pl, D, pl.diags[P.diag0].item0, "        ")
                  << "        fwd_diag_table<" << R << ", " << (D.has_rt ? "true" : "false") << ">(a, pg.tab + "
                  << op.diag * (1 << R) << ", c);\n      }\n";
                break;
            }
            default:
                break;
            }
        }
        if (last)
            o << "      fwd_scatter_global<" << R << ">(gb, gm, " << (st.has_phase ? "true" : "false")
              << ", dst, a, phase, kacc);\n";
        else
            o << "      fwd_scatter<T, " << K << ", " << R << ">(g, " << (st.has_phase ? "true" : "false")
              << ", tile, a, phase, kacc);\n"
              << "      __syncthreads();\n";
        o << "    }\n";
    }
    if (!dlast) o << "    IO::template store<NT>(tile, dst, base, row_off, tid);\n";
    // the next tile's first tile write must not overtake this tile's last tile reads
    if (P.n_stage > 1 || !dfirst || !dlast) o << "    __syncthreads();\n";
    o << "  }\n};\n} }\n"
      << "extern \"C\" __global__ void __launch_bounds__(" << NT << ", " << (NT >= 512 ? 1 : 2) << ") vqg_spec_fwd(" << kFwdArgs
      << ") {\n  vqg::fwd_pass_spec<float, " << K << ", " << R << ", vqg::spec::Body>(" << kFwdNames << ");\n}\n";
    return o.str();
}

// Shared-memory geometry of one specialised reverse pass: the program sized to the pass's
// own stages, ops, diagonal blocks and items (what load_prog copies), and two stash buffers
// of kMaxStageRows rows when they fit (one otherwise).
struct RevSpecGeo {
    int ops, stages, diags, items, rows;
    size_t smem;
};
RevSpecGeo rev_spec_geo(const Plan &pl, int pass) {
    const FPass &P = pl.passes[pass];
    RevSpecGeo g{};
    g.stages = std::max(1, (int)P.n_rstage);
    g.ops = 1;
    if (P.n_rstage) {
        const FStage &a = pl.stages[P.rstage0], &b = pl.stages[P.rstage0 + P.n_rstage - 1];
        g.ops = std::max(1, b.op0 + b.n_op - a.op0);
    }
    g.diags = std::max(1, (int)P.n_rdiag);
    g.items = 1;
    if (P.n_rdiag) {
        const FDiag &a = pl.diags[P.rdiag0], &b = pl.diags[P.rdiag0 + P.n_rdiag - 1];
        g.items = std::max(1, b.item0 + b.n_item - a.item0);
    }
    const size_t prog = prog_offsets(sizeof(float2), pl.Rr, g.stages, g.ops, g.diags, g.items).bytes;
    for (int rows : {2 * kMaxStageRows, kMaxStageRows}) {
        g.rows = rows;
        g.smem = rev_offsets(pl.K, pl.Rr, pl.L, sizeof(float2), sizeof(float), prog, rows).bytes;
        if (g.smem <= kMaxSmemBytes) break;
    }
    return g;
}

// Straight-line body of one reverse pass (mirrors rev_tile).
std::string gen_rev(const Plan &pl, int pass) {
    const FPass &P = pl.passes[pass];
    const int K = pl.K, R = pl.Rr, NT = 1 << (K - R);
    const int op_base = P.n_rstage ? pl.stages[P.rstage0].op0 : 0;
    const RevSpecGeo geo = rev_spec_geo(pl, pass);
    // with two stash buffers, consecutive reduction segments alternate between them: the
    // barrier before a segment's reduction also orders the reduction of the segment before
    // it (in the other buffer) ahead of that buffer's next writes, so no barrier follows
    // a reduction
    const bool dbuf = geo.rows == 2 * kMaxStageRows;
    int buf = 0;
    auto row_of = [&](int r) { return std::to_string(buf * kMaxStageRows + r); };
    auto buf_ptr = [&]() { return buf ? "stash + " + std::to_string(kMaxStageRows) + " * NT" : std::string("stash"); };
    std::ostringstream o;
    o << "#include \"fused_kernels.cuh\"\n"
      << "namespace vqg { namespace spec {\n"
      << "struct Body {\n"
      << "  static VQG_DEV void tile(float2 *tphi, float2 *tlam, const uint64_t *row_off, const Prog<float, " << R
      << "> &pg, uint64_t base, const float2 *__restrict__ phi_src, float2 *__restrict__ phi_dst, "
         "float2 *__restrict__ lam, double *acc, float *stash, int tid, bool write_phi, bool write_lam) {\n"
      << "    using T = float; using A = float2; using IO = TileIO<T, " << K << ">;\n"
      << "    constexpr int NT = " << NT << ", NA = " << (1 << R) << "; (void)NA;\n"
      << "    (void)row_off; (void)IO{};\n";
    const bool dfirst = P.n_rstage > 0 && direct_io(pl, P.rstage0, R);
    const bool dlast = P.n_rstage > 0 && direct_io(pl, P.rstage0 + P.n_rstage - 1, R);
    if (!dfirst)
        o << "    IO::template load2<NT, false>(tphi, phi_src, tlam, lam, base, row_off, tid);\n"
          << "    __syncthreads();\n";
    for (int s = 0; s < P.n_rstage; ++s) {
        const FStage &st = pl.stages[P.rstage0 + s];
        const bool first = s == 0 && dfirst, last = s == P.n_rstage - 1 && dlast;
        o << "    {  // stage " << s << "\n"
          << "      StageGeo<T, " << K << ", " << R << "> g; g.init(pg.st[" << s << "], tid, base);\n"
          << "      const uint64_t gb = g.gb; (void)gb;\n";
        if (first || last) o << "      " << gm_decl(pl, P.rstage0 + s, R) << "\n";
        if (first) o << "      A a[NA], l[NA]; rev_gather_global<" << R << ">(gb, gm, phi_src, lam, a, l);\n";
        else o << "      A a[NA], l[NA]; rev_gather<T, " << K << ", " << R << ">(g, tphi, tlam, a, l);\n";
        o << "      A phase = mk<T>((T)1, (T)0); T kacc = (T)1, k2acc = (T)1;\n";
        for (int i = 0; i < st.n_op; ++i) {
            const int oi = st.op0 + i, ol = oi - op_base;
            const FOp &op = pl.ops[oi];
            const std::string kb = std::to_string((int)op.k);
            const std::string srow = "stash[" + row_of((int)op.row) + " * NT + tid]";
            const std::string sptr = "stash + " + row_of((int)op.row) + " * NT + tid";
            switch (op.type) {
            case OP_RY:
                o << "      " << srow << " = rev_op_ry<" << kb << ", " << R << ", T>(a, l, " << prm(ol)
                  << ", kacc, k2acc);\n";
                break;
            case OP_RX:
                o << "      " << srow << " = rev_op_rx<" << kb << ", " << R << ", T>(a, l, " << prm(ol) << ", k2acc);\n";
                break;
            case OP_U3:
                o << "      rev_op_u3<" << kb << ", " << R << ", T>(a, l, " << prm(ol) << ", k2acc, " << sptr << ", NT);\n";
                break;
            case OP_CNOT:
                o << "      rev_op_cnot<" << kb << ", " << R << ", T>(a, l, " << op.rm0 << "u, "
                  << (op.rm0 ? std::string("false") : "(((gb >> " + std::to_string((int)op.cq) + ") & 1ull) != 0)")
                  << ");\n";
                break;
            case OP_CRX:
            case OP_CRY:
            case OP_CRZ:
            case OP_PH:
                o << "      " << srow << " = rev_op_cgen<" << (op.type - OP_CRX) << ", " << kb << ", " << R
                  << ", T>(a, l, " << prm(ol) << ", " << op.rm0 << "u, " << ctrl_expr(op) << ", k2acc);\n";
                break;
            case OP_DIAG: {
                // the block's own RZ items only, and the sign pattern only with a register-thread CZ
                const FDiag &D = pl.diags[P.rdiag0 + op.diag];
                o << "      {  // diagonal block " << op.diag << "\n";
                if (D.n_rz > 0) {
                    o << "        float H[" << R << "], S; rev_diag_sums<" << R << ">(a, l, H, S);\n";
                    for (int r = 0; r < D.n_rz; ++r) {
                        const FDItem &x = pl.items[D.item0 + r];
                        const std::string dst = "stash[" + row_of((int)op.row + r) + " * NT + tid]";
                        if (x.type == DI_RZ_REG)
                            o << "        " << dst << " = (2.f * H[" << x.k0 << "] - S) * k2acc;\n";
                        else
                            o << "        " << dst << " = ((gb & " << (unsigned long long)x.g0 << "ull) ? -S : S) * k2acc;\n";
                    }
                }
                o << diag_thread_code(pl, D, pl.diags[P.rdiag0].item0, "        ")
                  << "        rev_diag_table<" << R << ", " << (D.has_rt ? "true" : "false") << ">(a, l, pg.tab + "
                  << op.diag * (1 << R) << ", c);\n      }\n";
                break;
            }
            case OP_FLUSH:
                o << "      __syncthreads(); reduce_rows<T, NT>(" << buf_ptr() << ", " << op.lslot << ", " << (int)op.row
                  << ", acc, tid);" << (dbuf ? "" : " __syncthreads();") << "\n";
                if (dbuf) buf ^= 1;
                break;
            default:
                break;
            }
        }
        if (last)  // straight to HBM; the stash rows still need every thread's values
            o << "      rev_scatter_global<" << R << ">(gb, gm, " << (st.has_phase ? "true" : "false")
              << ", phi_dst, lam, write_phi, write_lam, a, l, phase, kacc);\n"
              << (st.n_rows ? "      __syncthreads();\n" : "");
        else
            o << "      rev_scatter<T, " << K << ", " << R << ">(g, " << (st.has_phase ? "true" : "false")
              << ", tphi, tlam, a, l, phase, kacc);\n"
              << "      __syncthreads();\n";
        if (st.n_rows) {
            o << "      reduce_stash<T, NT>(" << buf_ptr() << ", pg.st[" << s << "], acc, tid);"
              << (dbuf ? "" : " __syncthreads();") << "\n";
            if (dbuf) buf ^= 1;
        }
        o << "    }\n";
    }
    if (!dlast)
        o << "    if (write_phi) IO::template store<NT>(tphi, phi_dst, base, row_off, tid);\n"
          << "    if (write_lam) IO::template store<NT>(tlam, lam, base, row_off, tid);\n";
    // the next tile's first tile writes and stash rows must not overtake this tile's last
    // tile reads and reductions
    o << "    __syncthreads();\n"
      << "  }\n};\n} }\n"
      << "extern \"C\" __global__ void __launch_bounds__(" << NT << ") vqg_spec_rev(" << kRevArgs
      << ") {\n  using Caps = vqg::CapsT<" << geo.ops << ", " << geo.stages << ", " << geo.diags << ", " << geo.items
      << ">;\n"
      << "  // the launch passes this many bytes of dynamic shared memory (computed on the host)\n"
      << "  static_assert(vqg::RevCfg<float, " << K << ", " << R << ", Caps, " << geo.rows << ">::smem() == " << geo.smem
      << "ull, \"shared-memory size\");\n"
      << "  vqg::rev_pass_spec<float, " << K << ", " << R << ", vqg::spec::Body, Caps, " << geo.rows << ">("
      << kRevNames << ");\n}\n";
    return o.str();
}

uint64_t fnv1a(const std::string &x) {
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : x) h = (h ^ c) * 1099511628211ull;
    return h;
}

std::string dirname_of(const std::string &p) {
    const size_t k = p.find_last_of('/');
    return k == std::string::npos ? std::string(".") : p.substr(0, k);
}

// csrc and include directories next to the loaded libvqg.so
void source_dirs(std::string &csrc, std::string &inc) {
    Dl_info info;
    std::memset(&info, 0, sizeof info);
    dladdr((const void *)&fnv1a, &info);
    const std::string pkg = dirname_of(info.dli_fname ? info.dli_fname : "./libvqg.so");
    csrc = pkg + "/csrc";
    inc = dirname_of(pkg) + "/include";
    if (const char *e = std::getenv("VQG_SPEC_SRC")) csrc = e;  // headers kept elsewhere
    if (const char *e = std::getenv("VQG_SPEC_INC")) inc = e;
}

bool exists(const std::string &p) {
    struct stat sb;
    return stat(p.c_str(), &sb) == 0;
}

std::string nvcc_path() {
    if (const char *e = std::getenv("VQG_NVCC")) return e;
    if (const char *h = std::getenv("CUDA_HOME")) {
        const std::string p = std::string(h) + "/bin/nvcc";
        if (exists(p)) return p;
    }
    if (exists("/usr/local/cuda/bin/nvcc")) return "/usr/local/cuda/bin/nvcc";
    return "nvcc";
}

std::string cache_dir() {
    std::string d;
    if (const char *e = std::getenv("VQG_SPEC_CACHE")) d = e;
    else {
        const char *t = std::getenv("TMPDIR");
        d = std::string(t && *t ? t : "/tmp") + "/vqg_spec_" + std::to_string((long)getuid());
    }
    mkdir(d.c_str(), 0700);
    return d;
}

// Compile one source to a cubin unless the cache holds it; returns "" or an error text.
std::string compile_one(const std::string &src, const std::string &cubin, const std::string &base_cmd,
                        const std::string &dir) {
    if (exists(cubin)) return "";
    const std::string tag = std::to_string((long)getpid()) + "_" + std::to_string(fnv1a(cubin) & 0xffffff);
    const std::string cu = dir + "/src_" + tag + ".cu", tmp = dir + "/out_" + tag + ".cubin";
    {
        std::ofstream f(cu);
        f << src;
        if (!f) return "cannot write " + cu;
    }
    const std::string cmd = base_cmd + " -cubin -o '" + tmp + "' '" + cu + "' 2>&1";
    std::string out;
    FILE *pp = popen(cmd.c_str(), "r");
    if (!pp) return "cannot run " + cmd;
    char buf[512];
    while (fgets(buf, sizeof buf, pp)) out += buf;
    const int rc = pclose(pp);
    if (std::getenv("VQG_SPEC_KEEP")) std::rename(cu.c_str(), (cubin.substr(0, cubin.size() - 6) + ".cu").c_str());
    else std::remove(cu.c_str());
    if (rc != 0 || !exists(tmp)) {
        std::remove(tmp.c_str());
        if (out.size() > 1500) out = out.substr(out.size() - 1500);
        return "nvcc failed (" + std::to_string(rc) + "): " + out;
    }
    if (std::rename(tmp.c_str(), cubin.c_str()) != 0) return "cannot place " + cubin;
    return "";
}

std::mutex g_spec_mu;
std::map<std::string, cudaKernel_t> g_spec_kernels;  // cubin path -> kernel handle

int load_kernel(const std::string &cubin, const char *name, cudaKernel_t *out) {
    std::lock_guard<std::mutex> lock(g_spec_mu);
    auto it = g_spec_kernels.find(cubin);
    if (it != g_spec_kernels.end()) {
        *out = it->second;
        return VQG_OK;
    }
    std::ifstream f(cubin, std::ios::binary);
    std::vector<char> data((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
    if (data.empty()) return set_error(VQG_ERR_UNSUPPORTED, "specialised kernel %s is empty", cubin.c_str());
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, data.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    cudaKernel_t k = nullptr;
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&k, lib, name);
    if (e != cudaSuccess)
        return set_error(VQG_ERR_CUDA, "loading specialised kernel %s: %s", cubin.c_str(), cudaGetErrorString(e));
    g_spec_kernels[cubin] = k;
    *out = k;
    return VQG_OK;
}

size_t fwd_smem(int K, int R) {
#define VQG_S(KK, RR) if (K == KK && R == RR) return FwdCfg<float, KK, RR>::smem();
    VQG_S(10, 4) VQG_S(10, 5) VQG_S(11, 4) VQG_S(11, 5) VQG_S(12, 4) VQG_S(12, 5) VQG_S(13, 4) VQG_S(13, 5)
#undef VQG_S
    return 0;
}
size_t rev_smem(int K, int R) {
#define VQG_S(KK, RR) if (K == KK && R == RR) return RevCfg<float, KK, RR>::smem();
    VQG_S(10, 3) VQG_S(10, 4) VQG_S(11, 3) VQG_S(11, 4) VQG_S(12, 3) VQG_S(12, 4) VQG_S(13, 4)
#undef VQG_S
    return 0;
}

// Geometry of the Hamiltonian pass batches (HamGeo<float, K>): BA amplitudes per batch,
// D class bits at tile positions 0 (second amplitude of a chunk) and SH, SH + 1.
void ham_geo(int K, int &BA, int &D, int &SH) {
    const int chunks = (1 << K) / 2, cpt = chunks / 256, bch = std::min(cpt, 4);
    BA = 2 * bch;
    D = BA == 8 ? 3 : (BA == 4 ? 2 : (BA == 2 ? 1 : 0));
    SH = 4 + 5;
}
uint32_t class_bits(uint32_t zl, int D, int SH) {
    uint32_t c = 0;
    for (int d = 0; d < D; ++d) c |= ((zl >> (d == 0 ? 0 : SH + d - 1)) & 1u) << d;
    return c;
}
std::string hex(uint32_t v) {
    char b[16];
    std::snprintf(b, sizeof b, "0x%08xu", v);
    return b;
}

// Straight-line group work of one Hamiltonian pass (the arithmetic of ham_tile's group
// loop; every group takes the direct accumulation of its terms into the batch factors), in
// the slot order of ham_tile_spec: one 16-byte partner load per chunk and group.
std::string gen_ham(const Plan &pl, int h) {
    const HPass &P = pl.hp[h];
    const int K = pl.K;
    int BA, D, SH;
    ham_geo(K, BA, D, SH);
    const int BCH = BA / 2;
    const int term_base = P.n_group ? pl.hg[P.group0].term0 : 0;
    std::ostringstream o;
    o << "#include \"fused_kernels.cuh\"\n"
      << "namespace vqg { namespace spec {\n"
      << "struct Body {\n"
      << "  static VQG_DEV void groups(HamTab<float, " << K << "> &tb, const float2 *tile, uint32_t t0, "
      << "const uint32_t (&B)[" << BCH << "], const uint32_t (&b31)[" << BCH << "], const float2 (&mine)[" << BA
      << "], float2 (&delta)[" << BA << "]) {\n"
      << "    using A = float2; (void)b31; (void)tile; (void)B;\n";
    // A flip mask x splits into its bits at the batch's chunk positions (r: own chunk i
    // finds its partners in chunk i ^ r of the same batch), bit 0 (the slot inside a chunk)
    // and the rest y: the 16-byte loads q_k = tile[B[k] ^ (swz(y) & ~1)] depend on y alone,
    // so groups with the same y share them, and y = 0 needs none (the batch's own chunks).
    // The partner of slot j of chunk i is component j ^ (swz(x) & 1) of q_{i ^ r}.
    const uint32_t cmask = 1u | ((uint32_t)(BCH - 1) << SH);
    std::vector<int> order;  // the pass's groups, those with equal y adjacent
    {
        std::vector<uint32_t> ys;
        for (int g = 0; g < P.n_group; ++g) {
            const uint32_t y = pl.hg[P.group0 + g].xl & ~cmask;
            if (std::find(ys.begin(), ys.end(), y) == ys.end()) ys.push_back(y);
        }
        for (uint32_t y : ys)
            for (int g = 0; g < P.n_group; ++g)
                if ((pl.hg[P.group0 + g].xl & ~cmask) == y) order.push_back(g);
    }
    bool open = false;
    uint32_t cur_y = ~0u;
    for (int g : order) {
        const HGroup &G = pl.hg[P.group0 + g];
        if (G.n_term == 0) continue;  // the diagonal group exists even without terms
        const uint32_t y = G.xl & ~cmask, r = (G.xl >> SH) & (uint32_t)(BCH - 1);
        const uint32_t xs0 = swz<8>(G.xl) & 1u;
        if (y != cur_y) {
            if (open) o << "    }\n";
            o << "    {  // flip masks with y = " << hex(y) << "\n";
            if (y)
                for (int c = 0; c < BCH; ++c)
                    o << "      const float4 q" << c << " = *reinterpret_cast<const float4 *>(tile + (B[" << c << "] ^ "
                      << hex(swz<8>(y) & ~1u) << "));\n";
            open = true;
            cur_y = y;
        }
        // component pos of the partner chunk of own chunk i
        auto partner = [&](int i, int pos) {
            const int c = i ^ (int)r;
            if (!y) return "mine[" + std::to_string(2 * c + pos) + "]";
            const std::string q = "q" + std::to_string(c);
            return "make_float2(" + q + (pos ? ".z, " : ".x, ") + q + (pos ? ".w)" : ".y)");
        };
        const uint32_t x0 = xs0;
        bool re = true, im = true;
        for (int t = 0; t < G.n_term; ++t) {
            re = re && pl.ht[G.term0 + t].wi == 0.0;
            im = im && pl.ht[G.term0 + t].wr == 0.0;
        }
        const int kind = re ? 0 : (im ? 1 : 2);
        o << "      {  // group " << g << ": " << G.n_term << " term(s), kind " << kind << "\n";
        // the sign of slot j of chunk i for a term of class cls: parity((2i + j) & cls), a
        // literal, plus b_i where cls has bit 0
        auto neg = [](int i, int j, uint32_t cls) { return (__builtin_popcount((unsigned)(2 * i + j) & cls) & 1) != 0; };
        if (G.n_term == 1 && kind < 2) {
            const HTerm &t = pl.ht[G.term0];
            const uint32_t cls = class_bits(t.zl, D, SH);
            o << "      const A w = tb.g_w[" << g << "];\n"
              << "      const uint32_t wb = __float_as_uint(" << (kind == 0 ? "w.x" : "w.y") << ") ^ ((uint32_t)__popc(t0 & "
              << hex(t.zl) << ") << 31);\n";
            for (int i = 0; i < BCH; ++i) {
                o << "      { const uint32_t wi = wb" << ((cls & 1u) ? " ^ b31[" + std::to_string(i) + "]" : std::string()) << ";\n";
                for (int jj = 0; jj < 2; ++jj) {
                    const int k = 2 * i + jj;
                    o << "        { const float v = __uint_as_float(wi" << (neg(i, jj, cls) ? " ^ 0x80000000u" : "")
                      << "); const A p = " << partner(i, jj ^ (int)x0) << "; ";
                    if (kind == 0)
                        o << "delta[" << k << "].x = fmaf(v, p.x, delta[" << k << "].x); delta[" << k << "].y = fmaf(v, p.y, delta["
                          << k << "].y); }\n";
                    else
                        o << "delta[" << k << "].x = fmaf(-v, p.y, delta[" << k << "].x); delta[" << k << "].y = fmaf(v, p.x, delta["
                          << k << "].y); }\n";
                }
                o << "      }\n";
            }
        } else {
            o << "      float ux[" << BA << "], uy[" << BA << "];\n"
              << "      #pragma unroll\n      for (int k = 0; k < " << BA << "; ++k) ux[k] = 0.f, uy[k] = 0.f;\n";
            for (int t = 0; t < G.n_term; ++t) {
                const HTerm &tm = pl.ht[G.term0 + t];
                const int jt = G.term0 + t - term_base;
                const uint32_t cls = class_bits(tm.zl, D, SH);
                o << "      { const A w = tb.t_weff[" << jt << "]; const uint32_t s = (uint32_t)__popc(t0 & " << hex(tm.zl)
                  << ") << 31;";
                if (kind != 1) o << " const uint32_t bx = __float_as_uint(w.x) ^ s;";
                if (kind != 0) o << " const uint32_t by = __float_as_uint(w.y) ^ s;";
                o << "\n";
                for (int i = 0; i < BCH; ++i) {
                    const std::string bi = (cls & 1u) ? " ^ b31[" + std::to_string(i) + "]" : std::string();
                    for (int jj = 0; jj < 2; ++jj) {
                        const int k = 2 * i + jj;
                        const char *f = neg(i, jj, cls) ? " ^ 0x80000000u" : "";
                        o << "        ";
                        if (kind != 1) o << "ux[" << k << "] += __uint_as_float(bx" << bi << f << "); ";
                        if (kind != 0) o << "uy[" << k << "] += __uint_as_float(by" << bi << f << "); ";
                        o << "\n";
                    }
                }
                o << "      }\n";
            }
            for (int i = 0; i < BCH; ++i)
                for (int jj = 0; jj < 2; ++jj) {
                    const int k = 2 * i + jj;
                    o << "      { const A p = " << partner(i, jj ^ (int)x0) << "; ";
                    if (kind == 0)
                        o << "delta[" << k << "].x = fmaf(ux[" << k << "], p.x, delta[" << k << "].x); delta[" << k
                          << "].y = fmaf(ux[" << k << "], p.y, delta[" << k << "].y); }\n";
                    else if (kind == 1)
                        o << "delta[" << k << "].x = fmaf(-uy[" << k << "], p.y, delta[" << k << "].x); delta[" << k
                          << "].y = fmaf(uy[" << k << "], p.x, delta[" << k << "].y); }\n";
                    else
                        o << "delta[" << k << "] = cfma<float>(mk<float>(ux[" << k << "], uy[" << k << "]), p, delta[" << k
                          << "]); }\n";
                }
        }
        o << "      }\n";
    }
    if (open) o << "    }\n";
    o << "  }\n};\n} }\n"
      << "extern \"C\" __global__ void __launch_bounds__(256, 2) vqg_spec_ham(const float2 *__restrict__ psi, "
         "float2 *__restrict__ lam, const vqg::HPass *__restrict__ hp, int pi, const vqg::HGroup *__restrict__ groups, "
         "const vqg::HTerm *__restrict__ terms, uint64_t n_tiles, double *__restrict__ partials, int nb) {\n"
      << "  vqg::ham_pass_spec<float, " << K << ", vqg::spec::Body>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb);\n}\n";
    return o.str();
}

}  // namespace

// Generate and compile (in parallel, cached on disk) the specialised kernels of every pass
// of a complex64 plan: cubins[j] forward pass j and, with_rev, cubins[np + j] reverse pass
// j.  Host only.
// Compile sources to cubins in the cache directory (parallel, skipping cached ones).
int compile_sources(const std::vector<std::string> &srcs, std::vector<std::string> &cubins) {
    cubins.clear();
    std::string csrc, inc;
    source_dirs(csrc, inc);
    const std::string base_cmd = "'" + nvcc_path() +
                                 "' -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 "
                                 "--expt-relaxed-constexpr -I '" + csrc + "' -I '" + inc + "'";
    const std::string dir = cache_dir();
    // the cache key covers the generated source, the compiler command and the headers
    std::string headers;
    for (const char *h : {"fused_kernels.cuh", "fused.h", "df.cuh", "common.cuh", "kernels.h"}) {
        std::ifstream f(csrc + "/" + h);
        headers += std::string((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
    }
    const uint64_t hk = fnv1a(headers + base_cmd);
    for (const std::string &x : srcs) {
        char name[64];
        std::snprintf(name, sizeof name, "/%016llx_%016llx.cubin", (unsigned long long)fnv1a(x),
                      (unsigned long long)hk);
        cubins.push_back(dir + name);
    }
    std::vector<std::string> errs(srcs.size());
    const size_t nthr = std::max<size_t>(1, std::min<size_t>(srcs.size(), std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    std::mutex mu;
    size_t next = 0;
    for (size_t t = 0; t < nthr; ++t)
        pool.emplace_back([&] {
            for (;;) {
                size_t i;
                {
                    std::lock_guard<std::mutex> lock(mu);
                    if (next >= srcs.size()) return;
                    i = next++;
                }
                errs[i] = compile_one(srcs[i], cubins[i], base_cmd, dir);
            }
        });
    for (auto &th : pool) th.join();
    for (size_t i = 0; i < errs.size(); ++i)
        if (!errs[i].empty()) return set_error(VQG_ERR_UNSUPPORTED, "specialised kernel %zu: %s", i, errs[i].c_str());
    return VQG_OK;
}

int spec_compile(const Plan *pl, bool with_rev, std::vector<std::string> &cubins) {
    cubins.clear();
    if (!fwd_smem(pl->K, pl->Rf) || !rev_smem(pl->K, pl->Rr))
        return set_error(VQG_ERR_UNSUPPORTED, "no specialised kernels for K=%d Rf=%d Rr=%d", pl->K, pl->Rf, pl->Rr);
    const int np = (int)pl->passes.size();
    std::vector<std::string> srcs;
    for (int j = 0; j < np; ++j) srcs.push_back(gen_fwd(*pl, j));
    if (with_rev)
        for (int j = 0; j < np; ++j) srcs.push_back(gen_rev(*pl, j));
    return compile_sources(srcs, cubins);
}

size_t ham_smem(int K) {
    switch (K) {
    case 10: return HamCfg<float, 10>::smem();
    case 11: return HamCfg<float, 11>::smem();
    case 12: return HamCfg<float, 12>::smem();
    case 13: return HamCfg<float, 13>::smem();
    default: return 0;
    }
}

// The Hamiltonian passes of a complex64 plan: generate, compile, load.  The kernels belong
// to the plan's current Hamiltonian tables (recorded by their device address).
int spec_build_ham(Plan *pl) {
    pl->spec_ham.clear();
    pl->spec_ham_for = nullptr;
    const size_t sm = ham_smem(pl->K);
    if (!sm) return set_error(VQG_ERR_UNSUPPORTED, "no specialised Hamiltonian kernels for K=%d", pl->K);
    std::vector<std::string> srcs, cubins;
    for (int h = 0; h < (int)pl->hp.size(); ++h) srcs.push_back(gen_ham(*pl, h));
    if (int st = compile_sources(srcs, cubins)) return st;
    int dev = 0;
    cudaGetDevice(&dev);
    for (const std::string &c : cubins) {
        cudaKernel_t k = nullptr;
        if (int st = load_kernel(c, "vqg_spec_ham", &k)) return st;
        cudaError_t e = cudaKernelSetAttributeForDevice(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm, dev);
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "specialised kernel attribute: %s", cudaGetErrorString(e));
        pl->spec_ham.push_back((void *)k);
    }
    pl->spec_smem_ham = sm;
    pl->spec_ham_for = pl->d_hp;
    return VQG_OK;
}

int spec_launch_ham(const Plan *pl, int h, const void *psi, void *lam, double *partials, int nb, cudaStream_t s) {
    const float2 *a0 = (const float2 *)psi;
    float2 *a1 = (float2 *)lam;
    const HPass *a2 = pl->d_hp;
    int a3 = h;
    const HGroup *a4 = pl->d_hg;
    const HTerm *a5 = pl->d_ht;
    uint64_t a6 = pl->n_tiles;
    double *a7 = partials;
    int a8 = nb;
    void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8};
    return cudaLaunchKernel((const void *)pl->spec_ham[h], dim3(nb), dim3(256), args, pl->spec_smem_ham, s) ==
                   cudaSuccess ? VQG_OK : VQG_ERR_CUDA;
}

// spec_compile, then load every kernel for the current device.
int spec_build(Plan *pl, bool with_rev) {
    pl->spec_fwd.clear();
    pl->spec_rev.clear();
    std::vector<std::string> cubins;
    if (int st = spec_compile(pl, with_rev, cubins)) return st;
    const int np = (int)pl->passes.size();
    const size_t fsm = fwd_smem(pl->K, pl->Rf);
    pl->spec_smem_rev.clear();
    int dev = 0;
    cudaGetDevice(&dev);
    for (size_t i = 0; i < cubins.size(); ++i) {
        cudaKernel_t k = nullptr;
        const bool fwd = (int)i < np;
        // each reverse kernel's program and stash are sized for its own pass
        const size_t sm = fwd ? fsm : rev_spec_geo(*pl, (int)i - np).smem;
        if (int st = load_kernel(cubins[i], fwd ? "vqg_spec_fwd" : "vqg_spec_rev", &k)) return st;
        cudaError_t e = cudaKernelSetAttributeForDevice(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm, dev);
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "specialised kernel attribute: %s", cudaGetErrorString(e));
        (fwd ? pl->spec_fwd : pl->spec_rev).push_back((void *)k);
        if (!fwd) pl->spec_smem_rev.push_back(sm);
    }
    pl->spec_smem_fwd = fsm;
    return VQG_OK;
}

int spec_launch_fwd(const Plan *pl, int j, const void *src, void *dst, const void *mats, uint64_t n_tiles,
                    cudaStream_t s) {
    const float2 *a0 = (const float2 *)src;
    float2 *a1 = (float2 *)dst;
    const FPass *a2 = pl->d_passes;
    int a3 = j;
    const FStage *a4 = pl->d_stages;
    const FOp *a5 = pl->d_ops;
    const FDiag *a6 = pl->d_diags;
    const FDItem *a7 = pl->d_items;
    const float *a8 = (const float *)mats;
    uint64_t a9 = n_tiles;
    void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9};
    return cudaLaunchKernel((const void *)pl->spec_fwd[j], dim3(pl->grid_fwd), dim3(1 << (pl->K - pl->Rf)), args,
                            pl->spec_smem_fwd, s) == cudaSuccess ? VQG_OK : VQG_ERR_CUDA;
}

int spec_launch_rev(const Plan *pl, int j, const void *phi_src, void *phi_dst, void *lam, const void *mats,
                    double *partials, int nb, int wmask, uint64_t n_tiles, cudaStream_t s) {
    const float2 *a0 = (const float2 *)phi_src;
    float2 *a1 = (float2 *)phi_dst;
    float2 *a2 = (float2 *)lam;
    const FPass *a3 = pl->d_passes;
    int a4 = j;
    const FStage *a5 = pl->d_stages;
    const FOp *a6 = pl->d_ops;
    const FDiag *a7 = pl->d_diags;
    const FDItem *a8 = pl->d_items;
    const int *a9 = pl->d_slot_map;
    const float *a10 = (const float *)mats;
    uint64_t a11 = n_tiles;
    double *a12 = partials;
    int a13 = nb, a14 = wmask;
    void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9, &a10, &a11, &a12, &a13, &a14};
    return cudaLaunchKernel((const void *)pl->spec_rev[j], dim3(nb), dim3(1 << (pl->K - pl->Rr)), args,
                            pl->spec_smem_rev[j], s) == cudaSuccess ? VQG_OK : VQG_ERR_CUDA;
}

}  // namespace vqg

// Host-only: plan a circuit as vqg_circuit_create would with these options and compile
// the specialised kernels of its passes into the on-disk cache (no GPU is touched).
extern "C" int vqg_specialize_prepare(int n_qubits, const vqg_gate *gates, int n_gates, int n_params,
                                      const vqg_options *opt_in, int n_terms, const uint64_t *x_mask,
                                      const uint64_t *z_mask, const double *coef, int *n_kernels) {
    using namespace vqg;
    if (n_kernels) *n_kernels = 0;
    int st = vqg_validate_circuit(n_qubits, gates, n_gates, n_params, VQG_C64);
    if (st) return st;
    vqg_options opt;
    vqg_default_options(&opt);
    if (opt_in) opt = *opt_in;
    std::vector<vqg_gate> gv(gates, gates + n_gates);
    std::vector<int> slot_base(std::max(n_gates, 1), 0);
    int n_gslots = 0;
    for (int i = 0; i < n_gates; ++i) {
        slot_base[i] = n_gslots;
        n_gslots += reduce_values_of(gv[i].kind);
    }
    std::vector<HamGroup> ham;
    std::vector<PauliTerm> flat;
    if (n_terms > 0 && (st = group_pauli_terms(n_qubits, n_terms, x_mask, z_mask, coef, ham, flat))) return st;
    std::string err;
    Plan *pl = plan_gates(n_qubits, gv, slot_base, n_gslots, false, opt, err);
    if (!pl) return err.empty() ? VQG_OK : set_error(VQG_ERR_UNSUPPORTED, "%s", err.c_str());  // unfused: nothing
    std::vector<std::string> cubins, hcubins;
    st = spec_compile(pl, opt.specialize >= 2, cubins);
    if (!st && n_terms > 0 && plan_hamiltonian(pl, n_qubits, ham, flat)) {
        std::vector<std::string> srcs;
        for (int h = 0; h < (int)pl->hp.size(); ++h) srcs.push_back(gen_ham(*pl, h));
        st = compile_sources(srcs, hcubins);
    }
    delete pl;
    if (!st && n_kernels) *n_kernels = (int)(cubins.size() + hcubins.size());
    return st;
}
