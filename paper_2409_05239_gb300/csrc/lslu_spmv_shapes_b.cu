// Sparse products in the row shapes 8x1, 8x2 and 4x1 (lanes per row x chunks per step) (see lslu_spmv_impl.cuh),
// for the native vector type of each value type; selected per matrix by
// lslu_tune_spmv / lslu_set_spmv_shape.
#include "lslu_spmv_impl.cuh"

namespace lslu {

namespace {

template <int G, int U>
void run_shape(const DevCsr& A, int vt, const void* x, void* y, cudaStream_t s) {
  if (vt == LSLU_F64)
    spmv_run<double, double, double, G, U>(A, (const double*)x, (double*)y, s);
  else if (vt == LSLU_F32)
    spmv_run<float, float, float, G, U>(A, (const float*)x, (float*)y, s);
  else
    spmv_run<__nv_bfloat16, float, float, G, U>(A, (const float*)x, (float*)y, s);
}

template <int G, int U>
void run_shape_pivots(const DevCsr& A, int vt, const void* x, void* y, const PivotCoef& pc,
                      cudaStream_t s) {
  if (vt == LSLU_F64)
    spmv_pivots_run<double, double, double, G, U>(A, (const double*)x, (double*)y, pc, s);
  else if (vt == LSLU_F32)
    spmv_pivots_run<float, float, float, G, U>(A, (const float*)x, (float*)y, pc, s);
  else
    spmv_pivots_run<__nv_bfloat16, float, float, G, U>(A, (const float*)x, (float*)y, pc, s);
}

}  // namespace

void launch_spmv_shape_b(int shape, const DevCsr& A, int vt, const void* x, void* y, cudaStream_t s) {
  switch (shape) {
    case kShapeG8U1: run_shape<8, 1>(A, vt, x, y, s); break;
    case kShapeG8U2: run_shape<8, 2>(A, vt, x, y, s); break;
    case kShapeG4U1: run_shape<4, 1>(A, vt, x, y, s); break;
    default: break;
  }
}

void launch_spmv_pivots_shape_b(int shape, const DevCsr& A, int vt, const void* x, void* y,
                                const PivotCoef& pc, cudaStream_t s) {
  switch (shape) {
    case kShapeG8U1: run_shape_pivots<8, 1>(A, vt, x, y, pc, s); break;
    case kShapeG8U2: run_shape_pivots<8, 2>(A, vt, x, y, pc, s); break;
    case kShapeG4U1: run_shape_pivots<4, 1>(A, vt, x, y, pc, s); break;
    default: break;
  }
}

}  // namespace lslu
