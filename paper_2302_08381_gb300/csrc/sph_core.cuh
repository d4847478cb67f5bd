// Per-(l, m) assembly shared by every kernel family.
//
// arXiv 2302.08381, Eq. real-sh-cartesian with the prefactor folded into Q
// (Appendix C): Ytilde_l^0 = Qtilde_l^0 / sqrt2, Ytilde_l^{+m} = Qtilde_l^m c_m,
// Ytilde_l^{-m} = Qtilde_l^m s_m. Derivatives from Eq. iter-deri:
//   dQ/dx = x e Qtilde_{l-1}^{m+1},  dQ/dy = y e Qtilde_{l-1}^{m+1},
//   dQ/dz = f Qtilde_{l-1}^m,
//   dc_m/dx = m c_{m-1}, dc_m/dy = -m s_{m-1}, ds_m/dx = m s_{m-1}, ds_m/dy = m c_{m-1},
// and second derivatives by applying them twice:
//   d2Q/dx2 = e Qtilde_{l-1}^{m+1} + x^2 g2 Qtilde_{l-2}^{m+2},  d2Q/dxdy = x y g2 Qtilde_{l-2}^{m+2},
//   d2Q/dxdz = x g3 Qtilde_{l-2}^{m+1},  d2Q/dz2 = g4 Qtilde_{l-2}^m,
//   d2c_m/dx2 = m(m-1) c_{m-2}, d2c_m/dxdy = -m(m-1) s_{m-2}, d2c_m/dy2 = -m(m-1) c_{m-2},
//   d2s_m/dx2 = m(m-1) s_{m-2}, d2s_m/dxdy = m(m-1) c_{m-2}, d2s_m/dy2 = -m(m-1) s_{m-2}.
// The multipliers e, f, g2..g4 come from the host FP64 tables; those of the
// m = 0 column include the 1/sqrt2.
#pragma once

#include "sph_device.cuh"

namespace sph {

// Value, gradient and Hessian of one output column at one point.
template <typename T>
struct Deriv {
    T v;
    T gx, gy, gz;
    T hxx, hxy, hxz, hyy, hyz, hzz;
};

// Q-side quantities of channel m at degree l:
//   Q  = Qtilde_l^m, E1 = e Qtilde_{l-1}^{m+1}, Qz = f Qtilde_{l-1}^m,
//   G2 = g2 Qtilde_{l-2}^{m+2}, G3 = g3 Qtilde_{l-2}^{m+1}, G4 = g4 Qtilde_{l-2}^m.
template <typename T>
struct QParts {
    T Q, E1, Qz, G2, G3, G4;
};

// m = 0 column: C = 1 (the 1/sqrt2 is in the multipliers and in `inv_sqrt2`).
template <bool GRAD, bool HESS, typename T>
__device__ __forceinline__ Deriv<T> assemble_m0(const QParts<T>& q, T x, T y, T inv_sqrt2) {
    Deriv<T> d;
    d.v = q.Q * inv_sqrt2;
    if (GRAD || HESS) {
        d.gx = x * q.E1;
        d.gy = y * q.E1;
        d.gz = q.Qz;
    }
    if (HESS) {
        const T xg = x * q.G2, yg = y * q.G2;
        d.hxx = q.E1 + x * xg;
        d.hyy = q.E1 + y * yg;
        d.hxy = x * yg;
        d.hxz = x * q.G3;
        d.hyz = y * q.G3;
        d.hzz = q.G4;
    }
    return d;
}

// m > 0 columns. (cm, sm) = (c_m, s_m); (cm1, sm1) = (c_{m-1}, s_{m-1});
// (cm2, sm2) = (c_{m-2}, s_{m-2}) (unused when m = 1). `dc` receives the
// +m (cos-type) column, `ds` the -m (sin-type) column.
template <bool GRAD, bool HESS, typename T>
__device__ __forceinline__ void assemble_m(const QParts<T>& q, T x, T y, T mm, T mm1, T cm, T sm, T cm1,
                                           T sm1, T cm2, T sm2, Deriv<T>& dc, Deriv<T>& ds) {
    dc.v = q.Q * cm;
    ds.v = q.Q * sm;
    if (GRAD || HESS) {
        const T Qx = x * q.E1, Qy = y * q.E1;
        const T mQ = mm * q.Q;
        dc.gx = Qx * cm + mQ * cm1;
        dc.gy = Qy * cm - mQ * sm1;
        dc.gz = q.Qz * cm;
        ds.gx = Qx * sm + mQ * sm1;
        ds.gy = Qy * sm + mQ * cm1;
        ds.gz = q.Qz * sm;
        if (HESS) {
            const T Qxx = q.E1 + x * x * q.G2, Qyy = q.E1 + y * y * q.G2, Qxy = x * y * q.G2;
            const T Qxz = x * q.G3, Qyz = y * q.G3, Qzz = q.G4;
            const T mC = mm;                 // m
            const T m2 = mm * mm1;           // m (m - 1)
            // cos-type: C = c_m
            {
                const T Cx = mC * cm1, Cy = -mC * sm1;
                const T Cxx = m2 * cm2, Cxy = -m2 * sm2, Cyy = -m2 * cm2;
                dc.hxx = Qxx * cm + T(2) * Qx * Cx + q.Q * Cxx;
                dc.hyy = Qyy * cm + T(2) * Qy * Cy + q.Q * Cyy;
                dc.hzz = Qzz * cm;
                dc.hxy = Qxy * cm + Qx * Cy + Qy * Cx + q.Q * Cxy;
                dc.hxz = Qxz * cm + q.Qz * Cx;
                dc.hyz = Qyz * cm + q.Qz * Cy;
            }
            // sin-type: C = s_m
            {
                const T Cx = mC * sm1, Cy = mC * cm1;
                const T Cxx = m2 * sm2, Cxy = m2 * cm2, Cyy = -m2 * sm2;
                ds.hxx = Qxx * sm + T(2) * Qx * Cx + q.Q * Cxx;
                ds.hyy = Qyy * sm + T(2) * Qy * Cy + q.Q * Cyy;
                ds.hzz = Qzz * sm;
                ds.hxy = Qxy * sm + Qx * Cy + Qy * Cx + q.Q * Cxy;
                ds.hxz = Qxz * sm + q.Qz * Cx;
                ds.hyz = Qyz * sm + q.Qz * Cy;
            }
        }
    }
}

// Section 3's normalized harmonics are Ytilde evaluated at u = x/r. By the
// degree-l homogeneity of Ytilde (Euler), their Cartesian derivatives are
//   dY/dx_i     = (1/r) [g_i - l u_i Y]
//   d2Y/dxi dxj = (1/r^2) [H_ij - l (u_i g_j + u_j g_i) - l delta_ij Y + l (l+2) u_i u_j Y]
// with Y, g, H the value, gradient and Hessian of Ytilde at u.
template <bool HESS, typename T>
__device__ __forceinline__ void normalize_deriv(Deriv<T>& d, int l, T ux, T uy, T uz, T ir) {
    const T lf = T(l);
    const T lv = lf * d.v;
    const T gx = d.gx, gy = d.gy, gz = d.gz;
    if (HESS) {
        const T ir2 = ir * ir;
        const T c2 = lf * (lf + T(2)) * d.v;
        d.hxx = ir2 * (d.hxx - T(2) * lf * ux * gx - lv + c2 * ux * ux);
        d.hyy = ir2 * (d.hyy - T(2) * lf * uy * gy - lv + c2 * uy * uy);
        d.hzz = ir2 * (d.hzz - T(2) * lf * uz * gz - lv + c2 * uz * uz);
        d.hxy = ir2 * (d.hxy - lf * (ux * gy + uy * gx) + c2 * ux * uy);
        d.hxz = ir2 * (d.hxz - lf * (ux * gz + uz * gx) + c2 * ux * uz);
        d.hyz = ir2 * (d.hyz - lf * (uy * gz + uz * gy) + c2 * uy * uz);
    }
    d.gx = ir * (gx - ux * lv);
    d.gy = ir * (gy - uy * lv);
    d.gz = ir * (gz - uz * lv);
}

// Scale a point for the normalized form: u = xyz / r and r2 := |u|^2 as
// computed from the rounded u (0 at r = 0). Taking |u|^2 rather than exactly
// 1 keeps Q_l^m(z, r^2) the polynomial of the point u actually used; with
// r^2 = 1 the O(eps) mismatch is amplified ~l^2 times by Eq. iter-q. The
// chain rule of normalize_deriv is exact for any |u| (Euler's relation).
template <typename T>
__device__ __forceinline__ void unit_point(T& x, T& y, T& z, T& r2, T& ir) {
    const T rr = x * x + y * y + z * z;
    const T r = sqrt(rr);
    ir = (rr > T(0)) ? T(1) / r : T(0);
    x *= ir;
    y *= ir;
    z *= ir;
    r2 = x * x + y * y + z * z;
}

}  // namespace sph
