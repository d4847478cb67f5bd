// GENERATED by gen_hardcoded.py from the paper's Eqs. iter-sc, iter-q, Flm
// and real-sh-cartesian (Appendix C folding); do not edit by hand.
//
// hardcoded_l<LH>_<val|grad>(x, y, z, r2, vis, qa, qb) emits every column
// of degree l <= LH through vis.emit(l, k, Deriv) (k = l*l + l + m) and
// writes qa[m] = Qtilde_LH^m (m <= LH) and qb[m] = Qtilde_{LH-1}^m
// (m <= LH - 1), the state Eq. iter-q continues from at degree LH + 1.
#pragma once

#include "sph_core.cuh"

namespace sph {

// l <= 0, values: 0 operations after CSE.
template <typename T, typename Vis>
__device__ __forceinline__ void hardcoded_l0_val(T x, T y, T z, T r2, Vis& vis, T* qa, T* qb) {
    qa[0] = T(0.3989422804014327);
    {
        Deriv<T> d;
        d.v = T(0.28209479177387814);
        vis.emit(0, 0, d);
    }
}

// l <= 0, values and gradients: 0 operations after CSE.
template <typename T, typename Vis>
__device__ __forceinline__ void hardcoded_l0_grad(T x, T y, T z, T r2, Vis& vis, T* qa, T* qb) {
    qa[0] = T(0.3989422804014327);
    {
        Deriv<T> d;
        d.v = T(0.28209479177387814);
        d.gx = T(0);
        d.gy = T(0);
        d.gz = T(0);
        vis.emit(0, 0, d);
    }
}

// l <= 1, values: 4 operations after CSE.
template <typename T, typename Vis>
__device__ __forceinline__ void hardcoded_l1_val(T x, T y, T z, T r2, Vis& vis, T* qa, T* qb) {
    qb[0] = T(0.3989422804014327);
    qa[0] = T(0.690988298942671)*z;
    qa[1] = T(0.4886025119029199);
    {
        Deriv<T> d;
        d.v = T(0.28209479177387814);
        vis.emit(0, 0, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*y;
        vis.emit(1, 1, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*z;
        vis.emit(1, 2, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*x;
        vis.emit(1, 3, d);
    }
}

// l <= 1, values and gradients: 4 operations after CSE.
template <typename T, typename Vis>
__device__ __forceinline__ void hardcoded_l1_grad(T x, T y, T z, T r2, Vis& vis, T* qa, T* qb) {
    qb[0] = T(0.3989422804014327);
    qa[0] = T(0.690988298942671)*z;
    qa[1] = T(0.4886025119029199);
    {
        Deriv<T> d;
        d.v = T(0.28209479177387814);
        d.gx = T(0);
        d.gy = T(0);
        d.gz = T(0);
        vis.emit(0, 0, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*y;
        d.gx = T(0);
        d.gy = T(0.4886025119029199);
        d.gz = T(0);
        vis.emit(1, 1, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*z;
        d.gx = T(0);
        d.gy = T(0);
        d.gz = T(0.4886025119029199);
        vis.emit(1, 2, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*x;
        d.gx = T(0.4886025119029199);
        d.gy = T(0);
        d.gz = T(0);
        vis.emit(1, 3, d);
    }
}

// l <= 2, values: 20 operations after CSE.
template <typename T, typename Vis>
__device__ __forceinline__ void hardcoded_l2_val(T x, T y, T z, T r2, Vis& vis, T* qa, T* qb) {
    const T t0 = T(1.0925484305920792)*z;
    const T t1 = (z*z);
    qb[0] = T(0.690988298942671)*z;
    qb[1] = T(0.4886025119029199);
    qa[0] = -T(0.4460310290381928)*r2 + T(1.3380930871145784)*t1;
    qa[1] = t0;
    qa[2] = T(0.5462742152960396);
    {
        Deriv<T> d;
        d.v = T(0.28209479177387814);
        vis.emit(0, 0, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*y;
        vis.emit(1, 1, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*z;
        vis.emit(1, 2, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*x;
        vis.emit(1, 3, d);
    }
    {
        Deriv<T> d;
        d.v = T(1.0925484305920792)*x*y;
        vis.emit(2, 4, d);
    }
    {
        Deriv<T> d;
        d.v = t0*y;
        vis.emit(2, 5, d);
    }
    {
        Deriv<T> d;
        d.v = -T(0.31539156525252)*r2 + T(0.94617469575756)*t1;
        vis.emit(2, 6, d);
    }
    {
        Deriv<T> d;
        d.v = t0*x;
        vis.emit(2, 7, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.5462742152960396)*((x*x) - (y*y));
        vis.emit(2, 8, d);
    }
}

// l <= 2, values and gradients: 27 operations after CSE.
template <typename T, typename Vis>
__device__ __forceinline__ void hardcoded_l2_grad(T x, T y, T z, T r2, Vis& vis, T* qa, T* qb) {
    const T t0 = T(1.0925484305920792)*y;
    const T t1 = T(1.0925484305920792)*x;
    const T t2 = T(1.0925484305920792)*z;
    const T t3 = (z*z);
    qb[0] = T(0.690988298942671)*z;
    qb[1] = T(0.4886025119029199);
    qa[0] = -T(0.4460310290381928)*r2 + T(1.3380930871145784)*t3;
    qa[1] = t2;
    qa[2] = T(0.5462742152960396);
    {
        Deriv<T> d;
        d.v = T(0.28209479177387814);
        d.gx = T(0);
        d.gy = T(0);
        d.gz = T(0);
        vis.emit(0, 0, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*y;
        d.gx = T(0);
        d.gy = T(0.4886025119029199);
        d.gz = T(0);
        vis.emit(1, 1, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*z;
        d.gx = T(0);
        d.gy = T(0);
        d.gz = T(0.4886025119029199);
        vis.emit(1, 2, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*x;
        d.gx = T(0.4886025119029199);
        d.gy = T(0);
        d.gz = T(0);
        vis.emit(1, 3, d);
    }
    {
        Deriv<T> d;
        d.v = t0*x;
        d.gx = t0;
        d.gy = t1;
        d.gz = T(0);
        vis.emit(2, 4, d);
    }
    {
        Deriv<T> d;
        d.v = t0*z;
        d.gx = T(0);
        d.gy = t2;
        d.gz = t0;
        vis.emit(2, 5, d);
    }
    {
        Deriv<T> d;
        d.v = -T(0.31539156525252)*r2 + T(0.94617469575756)*t3;
        d.gx = -T(0.63078313050504)*x;
        d.gy = -T(0.63078313050504)*y;
        d.gz = T(1.26156626101008)*z;
        vis.emit(2, 6, d);
    }
    {
        Deriv<T> d;
        d.v = t1*z;
        d.gx = t2;
        d.gy = T(0);
        d.gz = t1;
        vis.emit(2, 7, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.5462742152960396)*((x*x) - (y*y));
        d.gx = t1;
        d.gy = -t0;
        d.gz = T(0);
        vis.emit(2, 8, d);
    }
}

// l <= 3, values: 44 operations after CSE.
template <typename T, typename Vis>
__device__ __forceinline__ void hardcoded_l3_val(T x, T y, T z, T r2, Vis& vis, T* qa, T* qb) {
    const T t0 = x*y;
    const T t1 = T(1.0925484305920792)*z;
    const T t2 = (z*z);
    const T t3 = (x*x);
    const T t4 = (y*y);
    const T t5 = t3 - t4;
    const T t6 = -T(0.4570457994644657)*r2 + T(2.2852289973223288)*t2;
    const T t7 = T(1.4453057213202771)*z;
    qb[0] = -T(0.4460310290381928)*r2 + T(1.3380930871145784)*t2;
    qb[1] = t1;
    qb[2] = T(0.5462742152960396);
    qa[0] = z*(-T(1.583253092116782)*r2 + T(2.63875515352797)*t2);
    qa[1] = t6;
    qa[2] = t7;
    qa[3] = T(0.5900435899266435);
    {
        Deriv<T> d;
        d.v = T(0.28209479177387814);
        vis.emit(0, 0, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*y;
        vis.emit(1, 1, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*z;
        vis.emit(1, 2, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*x;
        vis.emit(1, 3, d);
    }
    {
        Deriv<T> d;
        d.v = T(1.0925484305920792)*t0;
        vis.emit(2, 4, d);
    }
    {
        Deriv<T> d;
        d.v = t1*y;
        vis.emit(2, 5, d);
    }
    {
        Deriv<T> d;
        d.v = -T(0.31539156525252)*r2 + T(0.94617469575756)*t2;
        vis.emit(2, 6, d);
    }
    {
        Deriv<T> d;
        d.v = t1*x;
        vis.emit(2, 7, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.5462742152960396)*t5;
        vis.emit(2, 8, d);
    }
    {
        Deriv<T> d;
        d.v = y*(T(1.7701307697799304)*t3 - T(0.5900435899266435)*t4);
        vis.emit(3, 9, d);
    }
    {
        Deriv<T> d;
        d.v = T(2.8906114426405543)*t0*z;
        vis.emit(3, 10, d);
    }
    {
        Deriv<T> d;
        d.v = t6*y;
        vis.emit(3, 11, d);
    }
    {
        Deriv<T> d;
        d.v = z*(-T(1.1195289977703462)*r2 + T(1.865881662950577)*t2);
        vis.emit(3, 12, d);
    }
    {
        Deriv<T> d;
        d.v = t6*x;
        vis.emit(3, 13, d);
    }
    {
        Deriv<T> d;
        d.v = t5*t7;
        vis.emit(3, 14, d);
    }
    {
        Deriv<T> d;
        d.v = x*(T(0.5900435899266435)*t3 - T(1.7701307697799304)*t4);
        vis.emit(3, 15, d);
    }
}

// l <= 3, values and gradients: 79 operations after CSE.
template <typename T, typename Vis>
__device__ __forceinline__ void hardcoded_l3_grad(T x, T y, T z, T r2, Vis& vis, T* qa, T* qb) {
    const T t0 = T(1.0925484305920792)*y;
    const T t1 = T(1.0925484305920792)*x;
    const T t2 = T(1.0925484305920792)*z;
    const T t3 = (z*z);
    const T t4 = (x*x);
    const T t5 = (y*y);
    const T t6 = t4 - t5;
    const T t7 = x*y;
    const T t8 = T(3.540261539559861)*t7;
    const T t9 = T(1.7701307697799304)*t6;
    const T t10 = T(2.8906114426405543)*z;
    const T t11 = t10*y;
    const T t12 = t10*x;
    const T t13 = T(0.4570457994644657)*r2 - T(2.2852289973223288)*t3;
    const T t14 = -t13;
    const T t15 = -T(0.9140915989289314)*t7;
    const T t16 = y*z;
    const T t17 = T(1.1195289977703462)*r2;
    const T t18 = x*z;
    const T t19 = T(1.4453057213202771)*z;
    qb[0] = -T(0.4460310290381928)*r2 + T(1.3380930871145784)*t3;
    qb[1] = t2;
    qb[2] = T(0.5462742152960396);
    qa[0] = z*(-T(1.583253092116782)*r2 + T(2.63875515352797)*t3);
    qa[1] = t14;
    qa[2] = t19;
    qa[3] = T(0.5900435899266435);
    {
        Deriv<T> d;
        d.v = T(0.28209479177387814);
        d.gx = T(0);
        d.gy = T(0);
        d.gz = T(0);
        vis.emit(0, 0, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*y;
        d.gx = T(0);
        d.gy = T(0.4886025119029199);
        d.gz = T(0);
        vis.emit(1, 1, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*z;
        d.gx = T(0);
        d.gy = T(0);
        d.gz = T(0.4886025119029199);
        vis.emit(1, 2, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.4886025119029199)*x;
        d.gx = T(0.4886025119029199);
        d.gy = T(0);
        d.gz = T(0);
        vis.emit(1, 3, d);
    }
    {
        Deriv<T> d;
        d.v = t0*x;
        d.gx = t0;
        d.gy = t1;
        d.gz = T(0);
        vis.emit(2, 4, d);
    }
    {
        Deriv<T> d;
        d.v = t0*z;
        d.gx = T(0);
        d.gy = t2;
        d.gz = t0;
        vis.emit(2, 5, d);
    }
    {
        Deriv<T> d;
        d.v = -T(0.31539156525252)*r2 + T(0.94617469575756)*t3;
        d.gx = -T(0.63078313050504)*x;
        d.gy = -T(0.63078313050504)*y;
        d.gz = T(1.26156626101008)*z;
        vis.emit(2, 6, d);
    }
    {
        Deriv<T> d;
        d.v = t1*z;
        d.gx = t2;
        d.gy = T(0);
        d.gz = t1;
        vis.emit(2, 7, d);
    }
    {
        Deriv<T> d;
        d.v = T(0.5462742152960396)*t6;
        d.gx = t1;
        d.gy = -t0;
        d.gz = T(0);
        vis.emit(2, 8, d);
    }
    {
        Deriv<T> d;
        d.v = y*(T(1.7701307697799304)*t4 - T(0.5900435899266435)*t5);
        d.gx = t8;
        d.gy = t9;
        d.gz = T(0);
        vis.emit(3, 9, d);
    }
    {
        Deriv<T> d;
        d.v = t10*t7;
        d.gx = t11;
        d.gy = t12;
        d.gz = T(2.8906114426405543)*t7;
        vis.emit(3, 10, d);
    }
    {
        Deriv<T> d;
        d.v = t14*y;
        d.gx = t15;
        d.gy = -t13 - T(0.9140915989289314)*t5;
        d.gz = T(3.6563663957157257)*t16;
        vis.emit(3, 11, d);
    }
    {
        Deriv<T> d;
        d.v = z*(-t17 + T(1.865881662950577)*t3);
        d.gx = -T(2.2390579955406924)*t18;
        d.gy = -T(2.2390579955406924)*t16;
        d.gz = -t17 + T(3.3585869933110386)*t3;
        vis.emit(3, 12, d);
    }
    {
        Deriv<T> d;
        d.v = t14*x;
        d.gx = -t13 - T(0.9140915989289314)*t4;
        d.gy = t15;
        d.gz = T(3.6563663957157257)*t18;
        vis.emit(3, 13, d);
    }
    {
        Deriv<T> d;
        d.v = t19*t6;
        d.gx = t12;
        d.gy = -t11;
        d.gz = T(1.4453057213202771)*t6;
        vis.emit(3, 14, d);
    }
    {
        Deriv<T> d;
        d.v = x*(T(0.5900435899266435)*t4 - T(1.7701307697799304)*t5);
        d.gx = t9;
        d.gy = -t8;
        d.gz = T(0);
        vis.emit(3, 15, d);
    }
}

}  // namespace sph
