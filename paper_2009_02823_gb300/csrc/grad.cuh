// Gradient contraction shared by the finalize kernels.
#pragma once

#include <cuda_runtime.h>

namespace vqg {

// Contribution of U3 slot `slot` at occurrence with reduced sums o_rc (8 doubles at o):
// 2 Re sum_rc D_rc o_rc, D = (dU/dslot) U^dagger (App. B.1: one derivative per slot,
// all evaluated at the same point of the reverse sweep).
__device__ inline double u3_slot_contribution(const double *a, int slot, const double *o) {
    double s, c, sf, cf, sl, cl, sfl, cfl;
    sincos(0.5 * a[0], &s, &c);
    sincos(a[1], &sf, &cf);
    sincos(a[2], &sl, &cl);
    sincos(a[1] + a[2], &sfl, &cfl);
    // U (re, im)
    double u[4][2] = {{c, 0}, {-cl * s, -sl * s}, {cf * s, sf * s}, {cfl * c, sfl * c}};
    double d[4][2];
    if (slot == 0) {
        d[0][0] = -0.5 * s; d[0][1] = 0;
        d[1][0] = -cl * 0.5 * c; d[1][1] = -sl * 0.5 * c;
        d[2][0] = cf * 0.5 * c; d[2][1] = sf * 0.5 * c;
        d[3][0] = -cfl * 0.5 * s; d[3][1] = -sfl * 0.5 * s;
    } else if (slot == 1) {  // i e^{if} s, i e^{i(f+l)} c on the second row
        d[0][0] = 0; d[0][1] = 0; d[1][0] = 0; d[1][1] = 0;
        d[2][0] = -sf * s; d[2][1] = cf * s;
        d[3][0] = -sfl * c; d[3][1] = cfl * c;
    } else {  // -i e^{il} s, i e^{i(f+l)} c on the second column
        d[0][0] = 0; d[0][1] = 0;
        d[1][0] = sl * s; d[1][1] = -cl * s;
        d[2][0] = 0; d[2][1] = 0;
        d[3][0] = -sfl * c; d[3][1] = cfl * c;
    }
    // D = d * U^dagger, (U^dagger)_{kc} = conj(U_{ck})
    double acc = 0.0;
    for (int r = 0; r < 2; ++r)
        for (int cc = 0; cc < 2; ++cc) {
            double dr = 0, di = 0;
            for (int k = 0; k < 2; ++k) {
                const double *x = d[2 * r + k];
                const double ur = u[2 * cc + k][0], ui = -u[2 * cc + k][1];
                dr += x[0] * ur - x[1] * ui;
                di += x[0] * ui + x[1] * ur;
            }
            const double *orc = o + 2 * (2 * r + cc);
            acc += dr * orc[0] - di * orc[1];
        }
    return 2.0 * acc;
}

}  // namespace vqg
