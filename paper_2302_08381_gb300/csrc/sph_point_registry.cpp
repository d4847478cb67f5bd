// Table of the per-l_max POINT and batch-class launchers (one object file per l_max).
#include "sph_internal.h"

namespace sph {

#define SPH_DECL(L)                          \
    int point_fwd_L##L(const FwdArgs&);      \
    int point_bwd_L##L(const BwdArgs&);      \
    int point_dbwd_L##L(const BwdArgs&);     \
    int batch_class_L##L(const BatchClassArgs&);
SPH_DECL(0) SPH_DECL(1) SPH_DECL(2) SPH_DECL(3) SPH_DECL(4) SPH_DECL(5) SPH_DECL(6) SPH_DECL(7) SPH_DECL(8)
SPH_DECL(9) SPH_DECL(10) SPH_DECL(11) SPH_DECL(12) SPH_DECL(13) SPH_DECL(14) SPH_DECL(15) SPH_DECL(16)
#undef SPH_DECL

static_assert(SPH_MAX_L_POINT == 16, "registry lists l_max 0..16");

#define SPH_ROW(L) point_fwd_L##L
static const PointFwdFn kFwd[] = {SPH_ROW(0),  SPH_ROW(1),  SPH_ROW(2),  SPH_ROW(3),  SPH_ROW(4),  SPH_ROW(5),
                                  SPH_ROW(6),  SPH_ROW(7),  SPH_ROW(8),  SPH_ROW(9),  SPH_ROW(10), SPH_ROW(11),
                                  SPH_ROW(12), SPH_ROW(13), SPH_ROW(14), SPH_ROW(15), SPH_ROW(16)};
#undef SPH_ROW
#define SPH_ROW(L) point_bwd_L##L
static const PointBwdFn kBwd[] = {SPH_ROW(0),  SPH_ROW(1),  SPH_ROW(2),  SPH_ROW(3),  SPH_ROW(4),  SPH_ROW(5),
                                  SPH_ROW(6),  SPH_ROW(7),  SPH_ROW(8),  SPH_ROW(9),  SPH_ROW(10), SPH_ROW(11),
                                  SPH_ROW(12), SPH_ROW(13), SPH_ROW(14), SPH_ROW(15), SPH_ROW(16)};
#undef SPH_ROW
#define SPH_ROW(L) point_dbwd_L##L
static const PointBwdFn kDbwd[] = {SPH_ROW(0),  SPH_ROW(1),  SPH_ROW(2),  SPH_ROW(3),  SPH_ROW(4),  SPH_ROW(5),
                                   SPH_ROW(6),  SPH_ROW(7),  SPH_ROW(8),  SPH_ROW(9),  SPH_ROW(10), SPH_ROW(11),
                                   SPH_ROW(12), SPH_ROW(13), SPH_ROW(14), SPH_ROW(15), SPH_ROW(16)};
#undef SPH_ROW

#define SPH_ROW(L) batch_class_L##L
static const BatchClassFn kBatch[] = {SPH_ROW(0),  SPH_ROW(1),  SPH_ROW(2),  SPH_ROW(3),  SPH_ROW(4),  SPH_ROW(5),
                                      SPH_ROW(6),  SPH_ROW(7),  SPH_ROW(8),  SPH_ROW(9),  SPH_ROW(10), SPH_ROW(11),
                                      SPH_ROW(12), SPH_ROW(13), SPH_ROW(14), SPH_ROW(15), SPH_ROW(16)};
#undef SPH_ROW

int batch_one_gn0(const OneArgs&);
int batch_one_gn1(const OneArgs&);
int batch_one_gn2(const OneArgs&);
int batch_one_gn3(const OneArgs&);
static const BatchOneFn kOne[] = {batch_one_gn0, batch_one_gn1, batch_one_gn2, batch_one_gn3};
BatchOneFn batch_one_fn(int gn) { return (gn >= 0 && gn <= 3) ? kOne[gn] : nullptr; }

BatchClassFn batch_class_fn(int L) { return (L >= 0 && L <= SPH_MAX_L_POINT) ? kBatch[L] : nullptr; }
PointFwdFn point_fwd_fn(int L) { return (L >= 0 && L <= SPH_MAX_L_POINT) ? kFwd[L] : nullptr; }
PointBwdFn point_bwd_fn(int L) { return (L >= 0 && L <= SPH_MAX_L_POINT) ? kBwd[L] : nullptr; }
PointBwdFn point_dbwd_fn(int L) { return (L >= 0 && L <= SPH_MAX_L_POINT) ? kDbwd[L] : nullptr; }

size_t point_row_bytes(int L, int grad, int elem, int hess) {
    // Shared-memory bytes of one point's staged outputs: rows padded to an
    // odd stride when K is even (see RowStride in sph_point.cuh).
    const size_t K = size_t(L + 1) * size_t(L + 1);
    const bool pad = (K % 2 == 0);
    const size_t v = pad ? K + 1 : K, d = pad ? 3 * K + 1 : 3 * K, h = pad ? 9 * K + 1 : 9 * K;
    return size_t(elem) * (v + ((grad || hess) ? d : 0) + (hess ? h : 0));
}

}  // namespace sph
