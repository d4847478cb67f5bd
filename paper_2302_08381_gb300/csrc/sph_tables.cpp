// Host FP64 prefactor and recursion-coefficient tables.
//
// arXiv 2302.08381:
//  * Eq. Flm and Appendix C: F_l^0 = sqrt((2l+1)/(2 pi)),
//    F_l^m = -F_l^{m-1} / sqrt((l+m)(l+1-m)).
//  * Appendix C: the prefactor may be folded into Q, Qtilde_l^m = F_l^m Q_l^m,
//    which keeps every intermediate of the recursion O(1)-sized (Q_l^l alone
//    exceeds the FP32 range at l = 29 and F_l^l becomes subnormal there).
//  * Eq. iter-q rewritten for Qtilde:
//      Qtilde_l^l     = F_l^l Q_l^l with Q_l^l = -(2l-1) Q_{l-1}^{l-1}, Q_0^0 = 1
//      Qtilde_l^{l-1} = (2l-1) (F_l^{l-1}/F_{l-1}^{l-1}) z Qtilde_{l-1}^{l-1}
//      Qtilde_l^m     = a z Qtilde_{l-1}^m - b r^2 Qtilde_{l-2}^m,
//        a = (2l-1)/(l-m) F_l^m/F_{l-1}^m,  b = (l+m-1)/(l-m) F_l^m/F_{l-2}^m
//  * Eq. iter-deri rewritten for Qtilde:
//      dQtilde_l^m/dx = x e Qtilde_{l-1}^{m+1},  e = F_l^m/F_{l-1}^{m+1}
//      dQtilde_l^m/dz = f Qtilde_{l-1}^m,         f = (l+m) F_l^m/F_{l-1}^m
//    and, applied twice, the Hessian multipliers
//      g2 = F_l^m/F_{l-2}^{m+2}, g3 = (l+m) F_l^m/F_{l-2}^{m+1},
//      g4 = (l+m)(l+m-1) F_l^m/F_{l-2}^m.
//  The derivative multipliers of the m = 0 column carry the 1/sqrt2 of
//  Eq. real-sh-cartesian, so Ytilde_l^0 derivatives need no extra product.
//  * Eq. iter-q-alt (downward in m at fixed l; the printed form has the wrong
//    overall sign -- it gives Q_1^0 = -z -- and is used with the sign fixed):
//      Q_l^m = -[2(m+1) z Q_l^{m+1} + (x^2+y^2) Q_l^{m+2}] / ((l+m+1)(l-m)),
//    folded: Qtilde_l^m = al z Qtilde_l^{m+1} - be (x^2+y^2) Qtilde_l^{m+2},
//      al = -2(m+1)/((l+m+1)(l-m)) F_l^m/F_l^{m+1},
//      be = F_l^m/F_l^{m+2} / ((l+m+1)(l-m)),
//    started from Qtilde_l^l (with Qtilde_l^{l+1} = 0).
//  Q_l^l itself is never formed: Qtilde_l^l = -(2l-1)(F_l^l/F_{l-1}^{l-1}) Qtilde_{l-1}^{l-1}.
#include <cmath>
#include <mutex>

#include "sph_internal.h"

namespace sph {

namespace {

HostTables build_tables(int L) {
    HostTables t;
    t.lmax = L;
    const int n = tri_size(L);
    t.F.assign(n, 0.0);
    t.qll.assign(n, 0.0);
    t.d.assign(n, 0.0);
    t.a.assign(n, 0.0);
    t.b.assign(n, 0.0);
    t.e.assign(n, 0.0);
    t.fz.assign(n, 0.0);
    t.g2.assign(n, 0.0);
    t.g3.assign(n, 0.0);
    t.g4.assign(n, 0.0);
    t.al.assign(n, 0.0);
    t.be.assign(n, 0.0);
    t.inv_sqrt2 = 1.0 / std::sqrt(2.0);
    const double two_pi = 2.0 * 3.14159265358979323846;

    // Appendix C iteration for F_l^m.
    for (int l = 0; l <= L; ++l) {
        double f = std::sqrt((2.0 * l + 1.0) / two_pi);
        t.F[tri(l, 0)] = f;
        for (int m = 1; m <= l; ++m) {
            f = -f / std::sqrt(double(l + m) * double(l + 1 - m));
            t.F[tri(l, m)] = f;
        }
    }
    auto F = [&](int l, int m) -> double {
        if (l < 0 || m < 0 || m > l) return 0.0;
        return t.F[tri(l, m)];
    };
    auto ratio = [&](int l, int m, int l2, int m2) -> double {
        // F_l^m / F_l2^m2, zero when the denominator's Q vanishes (m2 > l2).
        if (l2 < 0 || m2 > l2 || m2 < 0) return 0.0;
        return F(l, m) / F(l2, m2);
    };

    // Qtilde_l^l by the folded form of Eq. iter-q's diagonal.
    double q = F(0, 0);
    t.qll[tri(0, 0)] = q;
    for (int l = 1; l <= L; ++l) {
        q = -(2.0 * l - 1.0) * ratio(l, l, l - 1, l - 1) * q;
        t.qll[tri(l, l)] = q;
    }
    for (int l = 1; l <= L; ++l) t.d[tri(l, l - 1)] = (2.0 * l - 1.0) * ratio(l, l - 1, l - 1, l - 1);

    for (int l = 0; l <= L; ++l) {
        for (int m = 0; m <= l; ++m) {
            const int i = tri(l, m);
            const double s0 = (m == 0) ? t.inv_sqrt2 : 1.0;
            if (m <= l - 2) {
                t.a[i] = (2.0 * l - 1.0) / double(l - m) * ratio(l, m, l - 1, m);
                t.b[i] = double(l + m - 1) / double(l - m) * ratio(l, m, l - 2, m);
                t.e[i] = s0 * ratio(l, m, l - 1, m + 1);
                t.g4[i] = s0 * double(l + m) * double(l + m - 1) * ratio(l, m, l - 2, m);
            }
            if (m <= l - 1) t.fz[i] = s0 * double(l + m) * ratio(l, m, l - 1, m);
            if (m <= l - 3) t.g3[i] = s0 * double(l + m) * ratio(l, m, l - 2, m + 1);
            if (m <= l - 4) t.g2[i] = s0 * ratio(l, m, l - 2, m + 2);
            const double den = double(l + m + 1) * double(l - m);
            if (m <= l - 1) t.al[i] = -2.0 * double(m + 1) / den * ratio(l, m, l, m + 1);
            if (m <= l - 2) t.be[i] = ratio(l, m, l, m + 2) / den;
        }
    }
    return t;
}

}  // namespace

const HostTables& host_tables() {
    static HostTables tables;
    static std::once_flag once;
    std::call_once(once, [] { tables = build_tables(SPH_MAX_L); });
    return tables;
}

}  // namespace sph
