// Tensor-core contraction interface (3xTF32 split complex operands, tcgen05).
#pragma once
#include <array>
#include <vector>

#include "tdmrg_internal.cuh"

namespace tdmrg {

// Planar split operand: float planes [4][nb][rows][ld] = re_hi, re_lo, im_hi, im_lo.
// K is the contraction extent (K-major rows), ld >= K a multiple of 4 floats, p 16-byte aligned.
struct TcOperand {
  float* p;
  int rows, K, ld, nb;
  long long plane() const { return (long long)nb * rows * ld; }
  long long floats() const { return 4 * plane(); }
};

inline int pad4(int k) { return (k + 3) & ~3; }

// C_b[m][n] = sum_{r < nred} sum_k opA(A[r*a_red + b*a_bat])[m][k] opB(B[r*b_red + b*b_bat])[n][k]
// with opX = conjugation when conjX.  out_mode 0: complex FP64 interleaved at
// C + b*sbc + m*ldc + n (double2 units); 1: FP32 planar (re at C + b*sbc + m*ldc + n, im at
// + plane); 2: split planes (4 planes of `plane` floats).
struct TcGemm {
  int M, N, K;
  int nred, nbatch;
  int a_red, a_bat, b_red, b_bat;
  int conjA, conjB;
  int out_mode;
  void* C;
  long long ldc, sbc, plane;
  int* status;
  // optional split-K scratch (FP32): when the output has few tiles, the (reduction x K) loop
  // is split over CTAs into partial sums that a second kernel adds up
  float* part;
  long long part_len;
  int ksplit;          // 0: tuned table / occupancy rule; > 0: forced (tc_gemm sets the one used)
  int bn;              // tile width: 0 = tuned table (else 64); 64 or 128 = forced
};

// g.ksplit on input: 0 = the tuned table's split for the shape (else the occupancy rule),
// > 0 = that split (capped by the K loop and the scratch); g.bn likewise for the tile width
cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, const TcGemm& g, cudaStream_t s);
// shapes (M, N, K, nred, nbatch) seen by tc_gemm while recording is on
void tc_record_shapes(bool on);
std::vector<std::array<int, 5>> tc_recorded_shapes();
// forget the loaded split-K table (read again at the next tc_gemm)
void tc_reload_table();
// the table's entry for a shape (host only, no CUDA call): false when the shape is not listed
bool tc_table_lookup(int M, int N, int K, int nred, int nbatch, int* ksplit, int* bn);
// dst(b, row, k) = conj?(src[b*sb + row*rs + k*ks])
cudaError_t split_f64(const cplx* src, long long sb, long long rs, long long ks, int conj,
                      const TcOperand& dst, cudaStream_t s);
// dst(b, row, k) = conj?(src[b*sb + k*kstride + row])   (tiled transpose)
cudaError_t split_f64_t(const cplx* src, long long sb, long long kstride, int conj,
                        const TcOperand& dst, cudaStream_t s);
// MPO mixing of an FP32 planar X[wi][a][s][t][b] into split planes.  trans 0: rows (a,s,t),
// K = b; trans 1: rows b, K = (a,s,t); trans 2: rows a, K = (s,t,b).
cudaError_t mix_split(const MixTable& T, int Ma, int d, int Mb, const float* X, long long xs,
                      long long xplane, const TcOperand& dst, int trans, cudaStream_t s);
cudaError_t planes_to_f64(const TcOperand& P, cplx* out, cudaStream_t s);

}  // namespace tdmrg
