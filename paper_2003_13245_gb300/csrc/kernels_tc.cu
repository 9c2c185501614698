// Tensor-core (tcgen05, sm_103a) complex contractions with 3xTF32 split products.
//
// A complex FP32 operand is stored as four planes: re_hi, re_lo, im_hi, im_lo, where
// x_hi = tf32(x) and x_lo = tf32(x - x_hi) (the split of Ootomo & Yokota); a real product
// x*y is taken as x_hi*y_hi + x_hi*y_lo + x_lo*y_hi with FP32 accumulation in tensor memory,
// and a complex product as four such real products (12 MMAs per 8-deep k step).
//
// One CTA computes a 128 x BN tile (BN = 64 or 128 columns, chosen per contraction shape by
// the tile table) of C = sum_r op(A_r) op(B_r)^T (both operands K-major).  Thread 0 issues the
// TMA loads (SWIZZLE_64B, 16-float = 64-byte rows, all four planes of a tile in one 4-D box),
// thread 32 issues tcgen05.mma into two TMEM accumulators (re, im: BN columns each), and all
// four warps read TMEM back with tcgen05.ld for the epilogue.  With 64-column tiles the stages
// are 48 KB: two per CTA when the grid has more CTAs than the GPU has SMs (two CTAs fit on an
// SM, so one's epilogue overlaps the other's main loop), four when it has at most one CTA per
// SM; 128-column tiles take three 64 KB stages.  Every wait is bounded and reports through
// `status`.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>

#include "tdmrg_internal.cuh"
#include "tc.cuh"

namespace tdmrg {

namespace {

constexpr int BM = 128;
constexpr int BK = 16;                          // floats per 64-byte swizzle row
constexpr int A_TILE = BM * BK * 4;             // one plane: 8 KB
// tile width BN = 64 or 128 columns: one B plane BN * 64 bytes; a stage holds the four planes
// of both operands (48 KB or 64 KB); TMEM holds the re accumulator in columns [0, BN) and the
// im accumulator in [BN, 2 BN)
__host__ __device__ constexpr int b_tile(int bn) { return bn * BK * 4; }
__host__ __device__ constexpr int stage_bytes(int bn) { return 4 * A_TILE + 4 * b_tile(bn); }
constexpr long long WAIT_CYCLES = 4000000000LL; // about 2 s
// pipeline depth: with 64-column tiles two stages when two CTAs share an SM (grids larger than
// the GPU), four when the grid leaves SMs with a single CTA; 128-column tiles take three
constexpr size_t smem_bytes(int nst, int bn) { return (size_t)nst * stage_bytes(bn) + 1024 + 256; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: false (and status set) after about 2 s
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(status, 3);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row atoms 512 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
  d |= (uint64_t)((8 * BK * 4) >> 4) << 32;        // stride byte offset: 8-row atoms
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)4 << 61;                          // SWIZZLE_64B
  return d;
}

// instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = bn
__host__ __device__ constexpr uint32_t idesc(int negA, int bn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)negA << 13) | ((uint32_t)(bn >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int NST, int BN>
__global__ void __launch_bounds__(128, NST == 2 ? 2 : 1)
    tc_zgemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    TcGemm g) {
  constexpr int B_TILE = b_tile(BN);
  constexpr int STAGE = stage_bytes(BN);
  constexpr int TMEM_COLS = 2 * BN;
  // the epilogue stages the re and im tiles (rows padded to BN + 1 floats) in the free stages
  static_assert(2 * BM * (BN + 1) * 4 <= NST * STAGE, "epilogue tile exceeds the stages");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * STAGE);
  uint64_t* empty = full + NST;
  uint64_t* done = empty + NST;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* s_issued = s_fail + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int ks = g.ksplit > 1 ? g.ksplit : 1;
  const int bz = blockIdx.z / ks, sp = blockIdx.z % ks;
  const int ktiles = (g.K + BK - 1) / BK;
  const int all = ktiles * g.nred;
  const int chunk = (all + ks - 1) / ks;
  const int tbeg = sp * chunk;
  const int tend = min(all, tbeg + chunk);
  const int total = tend > tbeg ? tend - tbeg : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *s_fail = 0;
    *s_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 0) {
    // producer
    for (int t = 0; t < total; ++t) {
      const int s = t % NST, use = t / NST;
      if (t >= NST && !mbar_wait(&empty[s], (use - 1) & 1, g.status)) {
        *s_fail = 1;
        break;
      }
      const int tt = tbeg + t;
      const int r = tt / ktiles, k0 = (tt % ktiles) * BK;
      unsigned char* st = smem + s * STAGE;
      mbar_expect_tx(&full[s], STAGE);
      tma_load_4d(st, &tmA, k0, m0, r * g.a_red + bz * g.a_bat, 0, &full[s]);
      tma_load_4d(st + 4 * A_TILE, &tmB, k0, n0, r * g.b_red + bz * g.b_bat, 0, &full[s]);
      *s_issued = t + 1;
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer.  Signs: Cr = Ar Br - (-1)^(cA+cB) Ai Bi, Ci = (-1)^cB Ar Bi + (-1)^cA Ai Br
    const int neg_ii = (g.conjA ^ g.conjB) ? 0 : 1;
    const int neg_ri = g.conjB;
    const int neg_ir = g.conjA;
    const uint32_t d_re = tmem, d_im = tmem + BN;
    bool first_re = true, first_im = true;
    int t = 0;
    for (; t < total; ++t) {
      const int s = t % NST;
      if (!mbar_wait(&full[s], (t / NST) & 1, g.status)) {
        *s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(smem + s * STAGE);
      const uint32_t b0 = a0 + 4 * A_TILE;
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        const uint32_t ko = kk * 32;
        const uint64_t arh = sdesc(a0 + 0 * A_TILE + ko), arl = sdesc(a0 + 1 * A_TILE + ko);
        const uint64_t aih = sdesc(a0 + 2 * A_TILE + ko), ail = sdesc(a0 + 3 * A_TILE + ko);
        const uint64_t brh = sdesc(b0 + 0 * B_TILE + ko), brl = sdesc(b0 + 1 * B_TILE + ko);
        const uint64_t bih = sdesc(b0 + 2 * B_TILE + ko), bil = sdesc(b0 + 3 * B_TILE + ko);
        // real part
        mma_tf32(d_re, arh, brh, idesc(0, BN), first_re ? 0u : 1u);
        first_re = false;
        mma_tf32(d_re, arh, brl, idesc(0, BN), 1u);
        mma_tf32(d_re, arl, brh, idesc(0, BN), 1u);
        mma_tf32(d_re, aih, bih, idesc(neg_ii, BN), 1u);
        mma_tf32(d_re, aih, bil, idesc(neg_ii, BN), 1u);
        mma_tf32(d_re, ail, bih, idesc(neg_ii, BN), 1u);
        // imaginary part
        mma_tf32(d_im, arh, bih, idesc(neg_ri, BN), first_im ? 0u : 1u);
        first_im = false;
        mma_tf32(d_im, arh, bil, idesc(neg_ri, BN), 1u);
        mma_tf32(d_im, arl, bih, idesc(neg_ri, BN), 1u);
        mma_tf32(d_im, aih, brh, idesc(neg_ir, BN), 1u);
        mma_tf32(d_im, aih, brl, idesc(neg_ir, BN), 1u);
        mma_tf32(d_im, ail, brh, idesc(neg_ir, BN), 1u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  // epilogue: every warp waits for the accumulators, then reads its 32 TMEM lanes
  const bool waited = mbar_wait(done, 0, g.status);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool ok = __syncthreads_and(waited ? 1 : 0) && !*s_fail;
  if (ok) {
    // TMEM -> registers -> shared tile (the pipeline stages are free now), then row-coalesced
    // global stores.  Tile rows are padded to 65 floats: conflict-free column writes.
    constexpr int TP = BN + 1;
    float* tre = reinterpret_cast<float*>(smem);
    float* tim = tre + BM * TP;
    const int lrow = warp * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
      float re[16], im[16];
      tmem_ld16(lane_addr + c, re);
      tmem_ld16(lane_addr + BN + c, im);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        tre[lrow * TP + c + i] = total == 0 ? 0.f : re[i];
        tim[lrow * TP + c + i] = total == 0 ? 0.f : im[i];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BM * BN; e += blockDim.x) {
      const int rl = e / BN, cl = e % BN;
      const int row = m0 + rl, n = n0 + cl;
      if (row >= g.M || n >= g.N) continue;
      const float vr = tre[rl * TP + cl], vi = tim[rl * TP + cl];
      if (ks > 1) {
        const long long pl = (long long)g.nbatch * ks * g.M * g.N;
        float* P = g.part + (((long long)bz * ks + sp) * g.M + row) * g.N;
        P[n] = vr;
        P[pl + n] = vi;
      } else if (g.out_mode == 0) {
        double2* C = reinterpret_cast<double2*>(g.C) + (long long)bz * g.sbc + (long long)row * g.ldc;
        C[n] = make_double2((double)vr, (double)vi);
      } else if (g.out_mode == 1) {
        float* Cr = reinterpret_cast<float*>(g.C) + (long long)bz * g.sbc + (long long)row * g.ldc;
        Cr[n] = vr;
        Cr[g.plane + n] = vi;
      } else {
        float* P = reinterpret_cast<float*>(g.C) + (long long)bz * g.sbc + (long long)row * g.ldc;
        const float rh = tf32_round(vr), ih = tf32_round(vi);
        P[n] = rh;
        P[g.plane + n] = tf32_round(vr - rh);
        P[2 * g.plane + n] = ih;
        P[3 * g.plane + n] = tf32_round(vi - ih);
      }
    }
  } else if (threadIdx.x == 0) {
    // a failed pipeline may still have copies in flight: wait (bounded) for the last load
    // issued into each stage before the shared memory is released
    const int issued = *s_issued;
    for (int s = 0; s < NST; ++s) {
      int last = -1;
      for (int t = s; t < issued; t += NST) last = t;
      if (last >= 0) mbar_wait(&full[s], (last / NST) & 1, g.status);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

// sum of the split-K partials into the requested output form
__global__ void split_reduce_kernel(TcGemm g) {
  const int ks = g.ksplit;
  const long long MN = (long long)g.M * g.N;
  const long long total = (long long)g.nbatch * MN;
  const long long pl = (long long)g.nbatch * ks * MN;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / MN);
    const long long mn = e % MN;
    const int row = (int)(mn / g.N), n = (int)(mn % g.N);
    float re = 0.f, im = 0.f;
    const float* P = g.part + (long long)b * ks * MN + mn;
    for (int s = 0; s < ks; ++s) {
      re += P[s * MN];
      im += P[pl + s * MN];
    }
    if (g.out_mode == 0) {
      double2* C = reinterpret_cast<double2*>(g.C) + (long long)b * g.sbc + (long long)row * g.ldc;
      C[n] = make_double2((double)re, (double)im);
    } else if (g.out_mode == 1) {
      float* Cr = reinterpret_cast<float*>(g.C) + (long long)b * g.sbc + (long long)row * g.ldc;
      Cr[n] = re;
      Cr[g.plane + n] = im;
    } else {
      float* Q = reinterpret_cast<float*>(g.C) + (long long)b * g.sbc + (long long)row * g.ldc;
      const float rh = tf32_round(re), ih = tf32_round(im);
      Q[n] = rh;
      Q[g.plane + n] = tf32_round(re - rh);
      Q[2 * g.plane + n] = ih;
      Q[3 * g.plane + n] = tf32_round(im - ih);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encoder() {
  if (g_encode) return cudaSuccess;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return cudaSuccess;
}

// 4-D map {K, rows, nb, 4 planes} with a {32, box_rows, 1, 4} box
cudaError_t make_map(CUtensorMap* m, const TcOperand& op, int box_rows) {
  if ((op.ld % 4) != 0 || op.ld < op.K || (reinterpret_cast<uintptr_t>(op.p) & 15) != 0)
    return cudaErrorInvalidValue;
  cuuint64_t dims[4] = {(cuuint64_t)op.K, (cuuint64_t)op.rows, (cuuint64_t)op.nb, 4};
  cuuint64_t strides[3] = {(cuuint64_t)op.ld * 4, (cuuint64_t)op.ld * 4 * op.rows,
                           (cuuint64_t)op.ld * 4 * op.rows * op.nb};
  cuuint32_t box[4] = {BK, (cuuint32_t)box_rows, 1, 4};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)op.p, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------------
// operand preparation
// ------------------------------------------------------------------------------------------
// dst planes [4][nb][rows][ld] from a complex FP64 source element (b, row, k) at
// src[b*sb + row*rs + k*ks] (conjugated if conj)
__global__ void split_f64_kernel(const double2* src, long long sb, long long rs, long long ks,
                                 int conj, float* dst, int nb, int rows, int K, int ld) {
  const long long plane = (long long)nb * rows * ld;
  const long long total = (long long)nb * rows * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % K);
    const long long r2 = e / K;
    const int row = (int)(r2 % rows);
    const int b = (int)(r2 / rows);
    double2 v = src[b * sb + row * rs + k * ks];
    const float re = (float)v.x, im = (float)(conj ? -v.y : v.y);
    const float rh = tf32_round(re), ih = tf32_round(im);
    const long long o = ((long long)b * rows + row) * ld + k;
    dst[o] = rh;
    dst[plane + o] = tf32_round(re - rh);
    dst[2 * plane + o] = ih;
    dst[3 * plane + o] = tf32_round(im - ih);
  }
}

// transposing variant through shared memory: dst(b, row, k) = src[b*sb + k*kstride + row]
// (the source is row-contiguous: consecutive rows are adjacent)
__global__ void split_f64_t_kernel(const double2* src, long long sb, long long kstride, int conj,
                                   float* dst, int nb, int rows, int K, int ld) {
  __shared__ double2 tile[32][33];
  const long long plane = (long long)nb * rows * ld;
  const int b = blockIdx.z;
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int k = k0 + yy, row = r0 + threadIdx.x;
    if (k < K && row < rows) tile[yy][threadIdx.x] = src[b * sb + (long long)k * kstride + row];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int row = r0 + yy, k = k0 + threadIdx.x;
    if (k < K && row < rows) {
      const double2 v = tile[threadIdx.x][yy];
      const float re = (float)v.x, im = (float)(conj ? -v.y : v.y);
      const float rh = tf32_round(re), ih = tf32_round(im);
      const long long o = ((long long)b * rows + row) * ld + k;
      dst[o] = rh;
      dst[plane + o] = tf32_round(re - rh);
      dst[2 * plane + o] = ih;
      dst[3 * plane + o] = tf32_round(im - ih);
    }
  }
}

// MPO channel mixing of an FP32 planar X[wi][a][u][t][b] (re plane, im plane at +xplane) into
// split planes.  trans 0: operand rows (a, s, t), K = b; trans 1: rows b, K = (a, s, t);
// trans 2: rows a, K = (s, t, b).  The block tables and FP32 operators are staged in shared
// memory; the inner loop is FP32 only.
constexpr int MIX_MAX_BLK = 64;
constexpr int MIX_MAX_OPS = 5000;     // float2 entries: nblk * d * d (40 KB)
__global__ void mix_split_kernel(int Dout, int Ma, int d, int Mb, const int* start,
                                 const int* chan, const float2* ops, int nblk, const float* X,
                                 long long xs, long long xplane, float* dst, int ld, int trans) {
  __shared__ float2 s_ops[MIX_MAX_OPS];
  __shared__ int s_start[MIX_MAX_BLK + 1];
  __shared__ int s_chan[MIX_MAX_BLK];
  for (int i = threadIdx.x; i < nblk * d * d; i += blockDim.x) s_ops[i] = ops[i];
  for (int i = threadIdx.x; i <= Dout; i += blockDim.x) s_start[i] = start[i];
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s_chan[i] = chan[i];
  __syncthreads();
  const long long per = (long long)Ma * d * d * Mb;
  const long long total = per * Dout;
  const int rows = trans == 1 ? Mb : (trans == 2 ? Ma : Ma * d * d);
  const long long plane = (long long)Dout * rows * ld;
  const long long ustride = (long long)d * Mb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    const int b = (int)(r % Mb); r /= Mb;
    const int tau = (int)(r % d); r /= d;
    const int sig = (int)(r % d); r /= d;
    const int a = (int)(r % Ma);
    const int wo = (int)(r / Ma);
    float ar = 0.f, ai = 0.f;
    for (int blk = s_start[wo]; blk < s_start[wo + 1]; ++blk) {
      const float2* op = s_ops + (blk * d + sig) * d;
      const float* x = X + s_chan[blk] * xs + ((long long)a * d * d + tau) * Mb + b;
      for (int u = 0; u < d; ++u) {
        const float2 o = op[u];
        if (o.x != 0.f || o.y != 0.f) {
          const float xr = x[u * ustride], xi = x[xplane + u * ustride];
          ar = fmaf(o.x, xr, fmaf(-o.y, xi, ar));
          ai = fmaf(o.x, xi, fmaf(o.y, xr, ai));
        }
      }
    }
    const int ast = (a * d + sig) * d + tau;
    long long o;
    if (trans == 1) o = ((long long)wo * rows + b) * ld + ast;
    else if (trans == 2) o = ((long long)wo * rows + a) * ld + (long long)(sig * d + tau) * Mb + b;
    else o = ((long long)wo * rows + ast) * ld + b;
    const float rh = tf32_round(ar), ih = tf32_round(ai);
    dst[o] = rh;
    dst[plane + o] = tf32_round(ar - rh);
    dst[2 * plane + o] = ih;
    dst[3 * plane + o] = tf32_round(ai - ih);
  }
}

// The same mixing with one thread per column (wo, a, tau, b) computing all D output levels
// sigma: the d input levels u of each block's channel are loaded once and reused for every
// sigma (the per-element form above reloads them d times).  The column index is decomposed in
// 32-bit arithmetic (the launcher checks that the columns number fewer than 2^31).
template <int D>
__global__ void __launch_bounds__(256, D >= 10 ? 2 : (D >= 8 ? 3 : 4)) mix_split_cols_kernel(int Dout, int Ma, int Mb,
                                                                const int* start, const int* chan,
                                                                const float2* ops, int nblk,
                                                                const float* X, long long xs,
                                                                long long xplane, float* dst,
                                                                int ld, int trans) {
  __shared__ float2 s_ops[MIX_MAX_OPS];
  __shared__ int s_start[MIX_MAX_BLK + 1];
  __shared__ int s_chan[MIX_MAX_BLK];
  for (int i = threadIdx.x; i < nblk * D * D; i += blockDim.x) s_ops[i] = ops[i];
  for (int i = threadIdx.x; i <= Dout; i += blockDim.x) s_start[i] = start[i];
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s_chan[i] = chan[i];
  __syncthreads();
  const int total = Dout * Ma * D * Mb;
  const int rows = trans == 1 ? Mb : (trans == 2 ? Ma : Ma * D * D);
  const long long plane = (long long)Dout * rows * ld;
  const long long ustride = (long long)D * Mb;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int r = e;
    const int b = r % Mb; r /= Mb;
    const int tau = r % D; r /= D;
    const int a = r % Ma;
    const int wo = r / Ma;
    float ar[D], ai[D];
#pragma unroll
    for (int sg = 0; sg < D; ++sg) ar[sg] = ai[sg] = 0.f;
    for (int blk = s_start[wo]; blk < s_start[wo + 1]; ++blk) {
      const float* x = X + s_chan[blk] * xs + ((long long)a * D * D + tau) * Mb + b;
      float xr[D], xi[D];
#pragma unroll
      for (int u = 0; u < D; ++u) {
        xr[u] = x[u * ustride];
        xi[u] = x[xplane + u * ustride];
      }
      const float2* op = s_ops + blk * D * D;
#pragma unroll
      for (int sg = 0; sg < D; ++sg)
#pragma unroll
        for (int u = 0; u < D; ++u) {
          const float2 o = op[sg * D + u];
          ar[sg] = fmaf(o.x, xr[u], fmaf(-o.y, xi[u], ar[sg]));
          ai[sg] = fmaf(o.x, xi[u], fmaf(o.y, xr[u], ai[sg]));
        }
    }
#pragma unroll
    for (int sg = 0; sg < D; ++sg) {
      const int ast = (a * D + sg) * D + tau;
      long long o;
      if (trans == 1) o = ((long long)wo * rows + b) * ld + ast;
      else if (trans == 2) o = ((long long)wo * rows + a) * ld + (long long)(sg * D + tau) * Mb + b;
      else o = ((long long)wo * rows + ast) * ld + b;
      const float rh = tf32_round(ar[sg]), ih = tf32_round(ai[sg]);
      dst[o] = rh;
      dst[plane + o] = tf32_round(ar[sg] - rh);
      dst[2 * plane + o] = ih;
      dst[3 * plane + o] = tf32_round(ai[sg] - ih);
    }
  }
}

// split planes (natural operand layout [4][nb][rows][ld]) -> complex FP64 [nb][rows][K]
__global__ void planes_to_f64_kernel(const float* P, int nb, int rows, int K, int ld,
                                     double2* out) {
  const long long plane = (long long)nb * rows * ld;
  const long long total = (long long)nb * rows * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % K);
    const long long br = e / K;
    const long long o = br * ld + k;
    out[e] = make_double2((double)P[o] + (double)P[plane + o],
                          (double)P[2 * plane + o] + (double)P[3 * plane + o]);
  }
}

// ---------------------------------------------------------------------------------------
// tile table: the split-K factor and the tile width (64 or 128 columns) of each contraction
// shape (M, N, K, nred, nbatch), measured by the tuning script shipped beside the library
// (tune_splitk.py) and read from tc_splitk_table.txt next to libtdmrg.so (or the file named
// by TDMRG_SPLITK_TABLE); a line "M N K nred nbatch ksplit [width]" (width 64 when absent).
// Shapes not in the table use 64-column tiles and the occupancy rule in tc_gemm.  Optionally
// every shape tc_gemm sees is recorded, which is how the tuning script learns the shapes of a
// workload.
// ---------------------------------------------------------------------------------------
using Shape = std::tuple<int, int, int, int, int>;
struct TileChoice {
  int ksplit = 0;
  int bn = 0;
};
std::mutex g_tab_mu;
bool g_tab_loaded = false;
std::map<Shape, TileChoice> g_tab;
bool g_record = false;
std::set<Shape> g_seen;

std::string table_path() {
  if (const char* p = std::getenv("TDMRG_SPLITK_TABLE")) return p;
  Dl_info info;
  if (dladdr(reinterpret_cast<void*>(&table_path), &info) && info.dli_fname) {
    std::string so = info.dli_fname;
    const size_t cut = so.find_last_of('/');
    return (cut == std::string::npos ? std::string(".") : so.substr(0, cut)) +
           "/tc_splitk_table.txt";
  }
  return "tc_splitk_table.txt";
}

void load_table_locked() {
  if (g_tab_loaded) return;
  g_tab_loaded = true;
  FILE* f = std::fopen(table_path().c_str(), "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    int M, N, K, r, b, ks, bn = 64;
    const int got = std::sscanf(line, "%d %d %d %d %d %d %d", &M, &N, &K, &r, &b, &ks, &bn);
    if (got >= 6 && ks >= 1 && (bn == 64 || bn == 128)) {
      TileChoice c;
      c.ksplit = ks;
      c.bn = got == 7 ? bn : 64;
      g_tab[Shape(M, N, K, r, b)] = c;
    }
  }
  std::fclose(f);
}

// the table's choice for a shape ({0, 0} when the shape is not listed)
TileChoice table_choice(const TcGemm& g) {
  std::lock_guard<std::mutex> lock(g_tab_mu);
  load_table_locked();
  const Shape key(g.M, g.N, g.K, g.nred, g.nbatch);
  if (g_record) g_seen.insert(key);
  const auto it = g_tab.find(key);
  return it == g_tab.end() ? TileChoice{} : it->second;
}

int grid_for(long long total) {
  long long b = (total + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, const TcGemm& g, cudaStream_t s) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  // once per process (the library serves one device): SM count and the kernels' attributes
  static std::once_flag once;
  static int n_sms = 0;
  static cudaError_t init_err = cudaSuccess;
  std::call_once(once, [] {
    int dev = 0, sms = 0;
    cudaError_t r = cudaGetDevice(&dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the largest shared-memory carveout, so that two 2-stage CTAs are resident per SM
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(tc_zgemm_kernel<2, 64>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(2, 64));
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(tc_zgemm_kernel<2, 64>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(tc_zgemm_kernel<4, 64>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(4, 64));
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(tc_zgemm_kernel<3, 128>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(3, 128));
    n_sms = sms;
    init_err = r;
  });
  if (init_err != cudaSuccess) return init_err;
  if (g.M < 1 || g.N < 1 || g.K < 1 || g.nred < 1 || g.nbatch < 1 || !g.status)
    return cudaErrorInvalidValue;
  if (g.bn != 0 && g.bn != 64 && g.bn != 128) return cudaErrorInvalidValue;
  if (A.K != g.K || B.K != g.K || A.rows < g.M || B.rows < g.N) return cudaErrorInvalidValue;
  // the batch / reduction coordinate of each operand must stay inside its nb
  const int amax = (g.nred - 1) * g.a_red + (g.nbatch - 1) * g.a_bat;
  const int bmax = (g.nred - 1) * g.b_red + (g.nbatch - 1) * g.b_bat;
  if (amax >= A.nb || bmax >= B.nb) return cudaErrorInvalidValue;
  // tile width and split-K: forced (timing), else the tuned table, else 64-column tiles and a
  // split when the output tiles cannot fill the GPU and the K loop is long
  const TileChoice tab = (g.ksplit > 0 && g.bn > 0) ? TileChoice{} : table_choice(g);
  const int bn = g.bn > 0 ? g.bn : (tab.bn > 0 ? tab.bn : 64);
  CUtensorMap ma, mb;
  if ((e = make_map(&ma, A, BM)) != cudaSuccess) return e;
  if ((e = make_map(&mb, B, bn)) != cudaSuccess) return e;
  TcGemm gg = g;
  gg.ksplit = 1;
  gg.bn = bn;
  const long long tiles = (long long)((g.N + bn - 1) / bn) * ((g.M + BM - 1) / BM) * g.nbatch;
  const int all = ((g.K + BK - 1) / BK) * g.nred;
  int ks = g.ksplit > 0 ? g.ksplit : tab.ksplit;
  if (ks == 0 && g.part && tiles < 76 && all >= 8) {
    ks = (int)((152 + tiles - 1) / tiles);
    if (ks > all / 4) ks = all / 4;
  }
  if (ks > all) ks = all;
  while (ks > 1 && (!g.part || 2LL * g.nbatch * ks * g.M * g.N > g.part_len)) --ks;
  if (ks > 1) gg.ksplit = ks;
  dim3 grid((g.N + bn - 1) / bn, (g.M + BM - 1) / BM, g.nbatch * gg.ksplit);
  count_launch();
  if (bn == 128)
    tc_zgemm_kernel<3, 128><<<grid, 128, smem_bytes(3, 128), s>>>(ma, mb, gg);
  else if ((long long)grid.x * grid.y * grid.z <= n_sms)
    tc_zgemm_kernel<4, 64><<<grid, 128, smem_bytes(4, 64), s>>>(ma, mb, gg);
  else
    tc_zgemm_kernel<2, 64><<<grid, 128, smem_bytes(2, 64), s>>>(ma, mb, gg);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (gg.ksplit > 1) {
    count_launch();
    split_reduce_kernel<<<grid_for((long long)g.nbatch * g.M * g.N), 256, 0, s>>>(gg);
    e = cudaGetLastError();
  }
  return e;
}

void tc_record_shapes(bool on) {
  std::lock_guard<std::mutex> lock(g_tab_mu);
  g_record = on;
  if (on) g_seen.clear();
}

std::vector<std::array<int, 5>> tc_recorded_shapes() {
  std::lock_guard<std::mutex> lock(g_tab_mu);
  std::vector<std::array<int, 5>> out;
  for (const auto& s : g_seen)
    out.push_back({std::get<0>(s), std::get<1>(s), std::get<2>(s), std::get<3>(s),
                   std::get<4>(s)});
  return out;
}

bool tc_table_lookup(int M, int N, int K, int nred, int nbatch, int* ksplit, int* bn) {
  std::lock_guard<std::mutex> lock(g_tab_mu);
  load_table_locked();
  const auto it = g_tab.find(Shape(M, N, K, nred, nbatch));
  if (it == g_tab.end()) return false;
  *ksplit = it->second.ksplit;
  *bn = it->second.bn;
  return true;
}

void tc_reload_table() {
  std::lock_guard<std::mutex> lock(g_tab_mu);
  g_tab.clear();
  g_tab_loaded = false;
}

cudaError_t split_f64(const cplx* src, long long sb, long long rs, long long ks, int conj,
                      const TcOperand& dst, cudaStream_t s) {
  const long long total = (long long)dst.nb * dst.rows * dst.K;
  count_launch();
  split_f64_kernel<<<grid_for(total), 256, 0, s>>>(src, sb, rs, ks, conj, dst.p, dst.nb, dst.rows,
                                                   dst.K, dst.ld);
  return cudaGetLastError();
}

cudaError_t split_f64_t(const cplx* src, long long sb, long long kstride, int conj,
                        const TcOperand& dst, cudaStream_t s) {
  dim3 grid((dst.rows + 31) / 32, (dst.K + 31) / 32, dst.nb);
  count_launch();
  split_f64_t_kernel<<<grid, dim3(32, 8), 0, s>>>(src, sb, kstride, conj, dst.p, dst.nb, dst.rows,
                                                  dst.K, dst.ld);
  return cudaGetLastError();
}

cudaError_t mix_split(const MixTable& T, int Ma, int d, int Mb, const float* X, long long xs,
                      long long xplane, const TcOperand& dst, int trans, cudaStream_t s) {
  const long long total = (long long)T.Dout * Ma * d * d * Mb;
  if (T.nblk > MIX_MAX_BLK || T.nblk * d * d > MIX_MAX_OPS || T.Dout > MIX_MAX_BLK)
    return cudaErrorInvalidValue;
  count_launch();
  const long long cols = (long long)T.Dout * Ma * d * Mb;
#define TDMRG_MIX_COLS(DD)                                                                    \
  case DD:                                                                                   \
    if (cols >= (1LL << 31) - 256LL * 152 * 32) break;                                       \
    mix_split_cols_kernel<DD><<<grid_for(cols), 256, 0, s>>>(T.Dout, Ma, Mb, T.start, T.chan, \
                                                             T.ops32, T.nblk, X, xs, xplane, \
                                                             dst.p, dst.ld, trans);          \
    return cudaGetLastError();
  switch (d) {
    TDMRG_MIX_COLS(2)
    TDMRG_MIX_COLS(3)
    TDMRG_MIX_COLS(4)
    TDMRG_MIX_COLS(5)
    TDMRG_MIX_COLS(6)
    TDMRG_MIX_COLS(7)
    TDMRG_MIX_COLS(8)
    TDMRG_MIX_COLS(9)
    TDMRG_MIX_COLS(10)
    default:
      break;
  }
#undef TDMRG_MIX_COLS
  mix_split_kernel<<<grid_for(total), 256, 0, s>>>(T.Dout, Ma, d, Mb, T.start, T.chan, T.ops32,
                                                   T.nblk, X, xs, xplane, dst.p, dst.ld, trans);
  return cudaGetLastError();
}

cudaError_t planes_to_f64(const TcOperand& P, cplx* out, cudaStream_t s) {
  const long long total = (long long)P.nb * P.rows * P.K;
  count_launch();
  planes_to_f64_kernel<<<grid_for(total), 256, 0, s>>>(P.p, P.nb, P.rows, P.K, P.ld, out);
  return cudaGetLastError();
}

}  // namespace tdmrg
