// Sparse products of Algorithm 4 with the matrix stream staged in shared
// memory by the Tensor Memory Accelerator (row shapes "tma" and
// "tma/16-bit").
//
// The CSR rows are cut into stages of whole rows (at most kTmaStageEntries
// padded entries and kTmaStageRows rows; host-side table, see lslu_spmv.cu).
// A persistent grid of about two blocks per SM splits the stages evenly.  In
// each block one thread keeps the next stages in flight with bulk copies
// (cp.async.bulk, completion counted on an mbarrier per ring slot) of the
// stage's values, columns (or 16-bit offsets and unit bases) and row
// pointers, while all threads consume the current stage: every thread takes
// 8-entry units (rows are padded to 8 entries, so a unit never straddles two
// rows), gathers x and forms the unit's dot product, then one thread per row
// adds its units' partials in order.  The DRAM stream therefore never waits
// for the gathers, and no registers hold it in flight.
//
// Order of the arithmetic (the same on every path, so results are bitwise
// reproducible and a pivot row computed by the pivot blocks equals its y
// entry): unit partial = FMAs over the unit's entries in order starting from
// 0; row value = 0 + the unit partials in order.
#include "lslu_spmv_impl.cuh"

namespace lslu {
namespace {

constexpr int kTmaThreads = 256;
constexpr int kTmaSlots = 4;  // ring of stages per block

template <typename VT>
constexpr int tma_stage_entries() {
  return sizeof(VT) == 8 ? kTmaStageEntriesF64 : kTmaStageEntries;
}

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }

// Shared-memory layout of one ring slot.
template <typename VT, bool CMP>
struct TmaSlot {
  static constexpr int SE = tma_stage_entries<VT>();
  static constexpr size_t vals = 0;
  static constexpr size_t cols = align128(vals + (size_t)SE * sizeof(VT));  // 32-bit columns
  static constexpr size_t offs = cols;                                       // or offsets
  static constexpr size_t ubase = align128(offs + (size_t)SE * 2);           // and unit bases
  static constexpr size_t rp =
      CMP ? align128(ubase + (size_t)(SE / 8 + 8) * 4) : align128(cols + (size_t)SE * 4);
  static constexpr size_t bytes = align128(rp + (size_t)(kTmaStageRows + 8) * 4);
};

template <typename VT, typename YT, bool CMP>
constexpr size_t tma_smem_bytes() {
  // header (mbarriers, stage descriptors), unit partials, ring slots
  return 256 + align128((size_t)(tma_stage_entries<VT>() / 8) * sizeof(YT)) +
         (size_t)kTmaSlots * TmaSlot<VT, CMP>::bytes;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false after kTmaWaitPolls unsuccessful polls
constexpr int kTmaWaitPolls = 1 << 20;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kTmaWaitPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Eight values of a unit (any state space) in the accumulation type.
template <typename YT>
__device__ __forceinline__ void unit_vals(const float* p, YT (&v)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = (YT)a.x; v[1] = (YT)a.y; v[2] = (YT)a.z; v[3] = (YT)a.w;
  v[4] = (YT)b.x; v[5] = (YT)b.y; v[6] = (YT)b.z; v[7] = (YT)b.w;
}
template <typename YT>
__device__ __forceinline__ void unit_vals(const double* p, YT (&v)[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 a = *reinterpret_cast<const double2*>(p + 2 * i);
    v[2 * i] = (YT)a.x;
    v[2 * i + 1] = (YT)a.y;
  }
}
template <typename YT>
__device__ __forceinline__ void unit_vals(const __nv_bfloat16* p, YT (&v)[8]) {
  const uint4 w = *reinterpret_cast<const uint4*>(p);
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = (YT)__uint_as_float(ws[i] << 16);
    v[2 * i + 1] = (YT)__uint_as_float(ws[i] & 0xffff0000u);
  }
}
__device__ __forceinline__ void unit_cols(const int32_t* p, int32_t (&c)[8]) {
  const int4 a = *reinterpret_cast<const int4*>(p);
  const int4 b = *reinterpret_cast<const int4*>(p + 4);
  c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
  c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
}
__device__ __forceinline__ void unit_cols(const uint16_t* p, int32_t base, int32_t (&c)[8]) {
  const uint4 w = *reinterpret_cast<const uint4*>(p);
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    c[2 * i] = base + (int32_t)(ws[i] & 0xffffu);
    c[2 * i + 1] = base + (int32_t)(ws[i] >> 16);
  }
}
template <typename YT, typename XT>
__device__ __forceinline__ YT unit_dot(const YT (&v)[8], const int32_t (&c)[8],
                                       const XT* __restrict__ x) {
  XT xv[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) xv[i] = __ldg(x + c[i]);
  YT acc = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) acc = fma(v[i], (YT)xv[i], acc);
  return acc;
}

struct TmaArgs {
  int64_t rows;
  const int32_t* row_ptr;  // padded entry offsets (rows + 1, readable to a multiple of 4)
  const int32_t* row_len;
  const int32_t* col;
  const uint16_t* off;
  const int32_t* ubase;    // readable to a multiple of 4 units
  const void* val;
  const int32_t* stage;    // 2 (nstages + 1): first row, first entry of every stage
  int nstages;
  int32_t* err;            // set to LSLU_ERR_TIMEOUT if a bounded wait gives up
};

// One CSR row in the order above, by one warp from global memory (every lane
// returns the value).
template <typename VT, typename XT, typename YT, bool CMP>
__device__ YT row_dot_units(int32_t row, const TmaArgs& t, const XT* __restrict__ x, int lane) {
  const int32_t start = __ldg(t.row_ptr + row), nu = __ldg(t.row_len + row) >> 3;
  const VT* val = reinterpret_cast<const VT*>(t.val);
  YT tot = 0;
  for (int32_t ub = 0; ub < nu; ub += 32) {
    const int32_t u = ub + lane;
    YT pu = 0;
    if (u < nu) {
      const int32_t p = start + u * 8;
      YT v[8];
      int32_t c[8];
      unit_vals<YT>(val + p, v);
      if constexpr (CMP)
        unit_cols(t.off + p, __ldg(t.ubase + (p >> 3)), c);
      else
        unit_cols(t.col + p, c);
      pu = unit_dot<YT, XT>(v, c, x);
    }
    const int cnt = min(32, nu - ub);
    for (int q = 0; q < cnt; ++q) tot += __shfl_sync(0xffffffffu, pu, q);
  }
  return tot;
}

template <typename VT, typename XT, typename YT, bool CMP>
__global__ void __launch_bounds__(kTmaThreads, 3)
    k_spmv_tma(TmaArgs t, const XT* __restrict__ x, YT* __restrict__ y, PivotCoef pc) {
  extern __shared__ __align__(128) unsigned char sm[];
  using Slot = TmaSlot<VT, CMP>;
  constexpr int SE = Slot::SE;
  const int npiv_all = pc.npiv_blocks * pc.nprob;
  if ((int)blockIdx.x < npiv_all) {
    pdl_wait();
    pdl_trigger();
    pivot_blocks<YT, 32>(pc, [=](int, int32_t row, int gl) {
      return row_dot_units<VT, XT, YT, CMP>(row, t, x, gl);
    });
    return;
  }
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm);            // kTmaSlots mbarriers
  int* desc = reinterpret_cast<int*>(sm + 64);                 // kTmaSlots x {r0, r1, e0, e1}
  YT* upart = reinterpret_cast<YT*>(sm + 256);                 // SE / 8 unit partials
  unsigned char* slots = sm + 256 + align128((size_t)(SE / 8) * sizeof(YT));
  const int tid = threadIdx.x;
  const int nb = (int)gridDim.x - npiv_all, b = (int)blockIdx.x - npiv_all;
  const int s0 = (int)((int64_t)b * t.nstages / nb), s1 = (int)((int64_t)(b + 1) * t.nstages / nb);
  const VT* val = reinterpret_cast<const VT*>(t.val);

  // the matrix and its stage table never change: the first stages are
  // requested before waiting for the kernel ahead
  auto issue = [&](int slot, int s) {
    const int r0 = __ldg(t.stage + 2 * s), e0 = __ldg(t.stage + 2 * s + 1);
    const int r1 = __ldg(t.stage + 2 * s + 2), e1 = __ldg(t.stage + 2 * s + 3);
    int* d = desc + 4 * slot;
    d[0] = r0; d[1] = r1; d[2] = e0; d[3] = e1;
    unsigned char* base = slots + (size_t)slot * Slot::bytes;
    const uint32_t bar = smem_u32(bars + slot);
    const uint32_t nv = (uint32_t)(e1 - e0) * (uint32_t)sizeof(VT);
    const int ra = r0 & ~3, rb = (r1 + 1 + 3) & ~3;
    const uint32_t nrp = (uint32_t)(rb - ra) * 4u;
    uint32_t ncol = 0, noff = 0, nub = 0;
    int ua = 0;
    if constexpr (CMP) {
      ua = (e0 >> 3) & ~3;
      const int ue = ((e1 >> 3) + 3) & ~3;
      noff = (uint32_t)(e1 - e0) * 2u;
      nub = (uint32_t)(ue - ua) * 4u;
    } else {
      ncol = (uint32_t)(e1 - e0) * 4u;
    }
    mbar_expect_tx(bar, nv + nrp + ncol + noff + nub);
    if (nv) bulk_g2s(smem_u32(base + Slot::vals), val + e0, nv, bar);
    if constexpr (CMP) {
      if (noff) bulk_g2s(smem_u32(base + Slot::offs), t.off + e0, noff, bar);
      if (nub) bulk_g2s(smem_u32(base + Slot::ubase), t.ubase + ua, nub, bar);
    } else {
      if (ncol) bulk_g2s(smem_u32(base + Slot::cols), t.col + e0, ncol, bar);
    }
    bulk_g2s(smem_u32(base + Slot::rp), t.row_ptr + ra, nrp, bar);
  };
  if (tid == 0) {
    for (int q = 0; q < kTmaSlots; ++q) mbar_init(smem_u32(bars + q), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < kTmaSlots && s0 + q < s1; ++q) issue(q, s0 + q);
  }
  __syncthreads();
  pdl_wait();  // x comes from the kernels before
  pdl_trigger();

  for (int i = 0; s0 + i < s1; ++i) {
    const int slot = i % kTmaSlots;
    const uint32_t parity = (uint32_t)(i / kTmaSlots) & 1u;
    const bool ok = mbar_wait(smem_u32(bars + slot), parity);
    const int* d = desc + 4 * slot;
    const int r0 = d[0], r1 = d[1], e0 = d[2], e1 = d[3];
    const unsigned char* base = slots + (size_t)slot * Slot::bytes;
    const VT* sv = reinterpret_cast<const VT*>(base + Slot::vals);
    const int nunits = (e1 - e0) >> 3;
    if (ok) {
      for (int u = tid; u < nunits; u += kTmaThreads) {
        YT v[8];
        int32_t c[8];
        unit_vals<YT>(sv + u * 8, v);
        if constexpr (CMP) {
          const uint16_t* so = reinterpret_cast<const uint16_t*>(base + Slot::offs);
          const int32_t* sb = reinterpret_cast<const int32_t*>(base + Slot::ubase);
          unit_cols(so + u * 8, sb[(e0 >> 3) + u - ((e0 >> 3) & ~3)], c);
        } else {
          unit_cols(reinterpret_cast<const int32_t*>(base + Slot::cols) + u * 8, c);
        }
        upart[u] = unit_dot<YT, XT>(v, c, x);
      }
    }
    if (__syncthreads_or(!ok)) {  // a copy never arrived: record it and leave together
      if (tid == 0) {
        atomicExch(t.err, LSLU_ERR_TIMEOUT);
        for (int p = 0; p < pc.nprob; ++p) atomicExch(&pc.st[p].status, LSLU_ERR_TIMEOUT);
        for (int q = 0; q < kTmaSlots && s0 + i + q < s1; ++q)  // copies still in flight
          mbar_wait(smem_u32(bars + (i + q) % kTmaSlots), (uint32_t)((i + q) / kTmaSlots) & 1u);
      }
      return;
    }
    {
      const int32_t* srp = reinterpret_cast<const int32_t*>(base + Slot::rp);
      const int ra = r0 & ~3;
      for (int r = r0 + tid; r < r1; r += kTmaThreads) {
        const int ua = (srp[r - ra] - e0) >> 3, ub = (srp[r + 1 - ra] - e0) >> 3;
        YT tot = 0;
        for (int u = ua; u < ub; ++u) tot += upart[u];
        y[r] = tot;
      }
    }
    __syncthreads();  // the slot and the partials are free
    if (tid == 0 && s0 + i + kTmaSlots < s1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(slot, s0 + i + kTmaSlots);
    }
  }
  (void)SE;
}

template <typename VT, typename XT, typename YT, bool CMP>
void run_tma(const DevCsr& A, const XT* x, YT* y, PivotCoef pc, cudaStream_t s) {
  constexpr size_t smem = tma_smem_bytes<VT, YT, CMP>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_spmv_tma<VT, XT, YT, CMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  TmaArgs t{A.rows, A.row_ptr, A.row_len, A.col, A.off, A.ubase, A.val, A.tma_stage,
            A.tma_nstages, A.tma_err};
  const int nstream = std::max(1, std::min(A.tma_blocks, A.tma_nstages));
  const int64_t blocks = (int64_t)pc.npiv_blocks * pc.nprob + nstream;
  launch_pdl(k_spmv_tma<VT, XT, YT, CMP>, dim3((unsigned)blocks), dim3(kTmaThreads), smem, s, t,
             x, y, pc);
}

template <typename VT, typename XT, typename YT>
void run_tma_fmt(const DevCsr& A, const XT* x, YT* y, const PivotCoef& pc, cudaStream_t s) {
  if (A.use_cmp)
    run_tma<VT, XT, YT, true>(A, x, y, pc, s);
  else
    run_tma<VT, XT, YT, false>(A, x, y, pc, s);
}

}  // namespace

size_t tma_smem_need(int vt, int cmp) {
  if (vt == LSLU_F64)
    return cmp ? tma_smem_bytes<double, double, true>() : tma_smem_bytes<double, double, false>();
  if (vt == LSLU_F32)
    return cmp ? tma_smem_bytes<float, float, true>() : tma_smem_bytes<float, float, false>();
  return cmp ? tma_smem_bytes<__nv_bfloat16, float, true>()
             : tma_smem_bytes<__nv_bfloat16, float, false>();
}

// Products of the staged shapes in the native vector type (FP64 for FP64
// values, FP32 otherwise); pc.npiv_blocks = 0 for a plain product.
void launch_spmv_pivots_tma(const DevCsr& A, int vt, const void* x, void* y, const PivotCoef& pc,
                            cudaStream_t s) {
  if (A.rows == 0 || !A.tma_ok) return;
  if (vt == LSLU_F64)
    run_tma_fmt<double, double, double>(A, (const double*)x, (double*)y, pc, s);
  else if (vt == LSLU_F32)
    run_tma_fmt<float, float, float>(A, (const float*)x, (float*)y, pc, s);
  else
    run_tma_fmt<__nv_bfloat16, float, float>(A, (const float*)x, (float*)y, pc, s);
}

void launch_spmv_tma(const DevCsr& A, int vt, const void* x, void* y, cudaStream_t s) {
  PivotCoef pc = {};
  pc.npiv_blocks = 0;
  pc.nprob = 0;
  launch_spmv_pivots_tma(A, vt, x, y, pc, s);
}

}  // namespace lslu
