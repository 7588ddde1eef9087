// Sparse products in the warp-per-row stride-1 shapes 32x8e and 32x4e (32
// lanes on consecutive entries of a row, 8 or 4 entries in flight per lane;
// see row_dot_s1 in lslu_spmv_impl.cuh), for the native vector type of each
// value type; selected per matrix by lslu_tune_spmv / lslu_set_spmv_shape.
#include "lslu_spmv_impl.cuh"

namespace lslu {

namespace {

template <int U>
void run_shape(const DevCsr& A, int vt, const void* x, void* y, cudaStream_t s) {
  if (vt == LSLU_F64)
    spmv_run<double, double, double, 0, U>(A, (const double*)x, (double*)y, s);
  else if (vt == LSLU_F32)
    spmv_run<float, float, float, 0, U>(A, (const float*)x, (float*)y, s);
  else
    spmv_run<__nv_bfloat16, float, float, 0, U>(A, (const float*)x, (float*)y, s);
}

template <int U>
void run_shape_pivots(const DevCsr& A, int vt, const void* x, void* y, const PivotCoef& pc,
                      cudaStream_t s) {
  if (vt == LSLU_F64)
    spmv_pivots_run<double, double, double, 0, U>(A, (const double*)x, (double*)y, pc, s);
  else if (vt == LSLU_F32)
    spmv_pivots_run<float, float, float, 0, U>(A, (const float*)x, (float*)y, pc, s);
  else
    spmv_pivots_run<__nv_bfloat16, float, float, 0, U>(A, (const float*)x, (float*)y, pc, s);
}

}  // namespace

void launch_spmv_shape_c(int shape, const DevCsr& A, int vt, const void* x, void* y,
                         cudaStream_t s) {
  if (shape == kShapeE8 || shape == kShapeE8Cmp)
    run_shape<8>(A, vt, x, y, s);
  else
    run_shape<4>(A, vt, x, y, s);
}

void launch_spmv_pivots_shape_c(int shape, const DevCsr& A, int vt, const void* x, void* y,
                                const PivotCoef& pc, cudaStream_t s) {
  if (shape == kShapeE8 || shape == kShapeE8Cmp)
    run_shape_pivots<8>(A, vt, x, y, pc, s);
  else
    run_shape_pivots<4>(A, vt, x, y, pc, s);
}

}  // namespace lslu
