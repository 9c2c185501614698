// TDVP engine: device storage, the contraction building blocks and the one-site
// projector-splitting sweep (imaginary and real time), the variational application of the
// current MPO and the MPS-MPO-MPS overlap.
#include "engine.h"
#include "tc.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <exception>
#include <string>
#include <thread>

#include "../../include/tdmrg.h"

namespace tdmrg {

namespace {
constexpr long long NOSPLIT = 1LL << 60;
// gauge-QR rank threshold of the mixed path (a larger threshold, at the 3xTF32 noise level,
// changes neither C(t) nor log Z measurably but sends many columns through completion)
constexpr double kMixedRankTol = 1e-12;
const cplx ONE = {1.0, 0.0};
const cplx ZERO = {0.0, 0.0};

MatRef mref(const cplx* p, long long rs, long long cs, long long sb = 0, long long sr = 0,
            int conj = 0) {
  MatRef r;
  r.p = p;
  r.rs = rs;
  r.cs = cs;
  r.sb = sb;
  r.sr = sr;
  r.conj = conj;
  return r;
}
QrRef qref(const cplx* p, long long rs, long long cs, long long cb, long long cbs, int conj) {
  QrRef r;
  r.p = p;
  r.rs = rs;
  r.cs = cs;
  r.cb = cb;
  r.cbs = cbs;
  r.conj = conj;
  return r;
}
}  // namespace

void throw_cuda(cudaError_t e, const char* what, int line) {
  const int code = (e == cudaErrorMemoryAllocation) ? TDMRG_ERR_OOM : TDMRG_ERR_CUDA;
  throw Failure{code, std::string(cudaGetErrorString(e)) + " in " + what + " (engine.cu:" +
                          std::to_string(line) + ")"};
}

// ------------------------------------------------------------------------------------
// contraction building blocks
// ------------------------------------------------------------------------------------
void heff_f64(const Ctx& c, const DevMpoSite& W, int Ml, int Mr, int D, int d, const cplx* Lenv,
              const cplx* Renv, const cplx* in, cplx* out, const int* skip) {
  const long long per = (long long)Ml * D * Mr;
  // X[(w,a)][(s,c)] = sum_y L[w,a,y] in[y,(s,c)]
  CK(zgemm(W.Dl * Ml, D * Mr, Ml, 1, 1, ONE, mref(Lenv, Ml, 1), mref(in, (long long)D * Mr, 1),
           ZERO, c.X, (long long)D * Mr, 0, skip, c.st));
  // Y[v][a][s][t][c] = sum_{w,u} W[w,v,s,u] X[w][a][u][t][c]
  CK(mpo_mix(W.lr, Ml, d, Mr, c.X, per, c.Y, per, skip, c.st));
  // out[(a,s)][b] = sum_{v,c} Y[v][(a,s)][c] R[v][b][c]
  CK(zgemm(Ml * D, Mr, Mr, 1, W.Dr, ONE, mref(c.Y, Mr, 1, 0, per),
           mref(Renv, 1, Mr, 0, (long long)Mr * Mr), ZERO, out, Mr, 0, skip, c.st));
}

void left_partial_f64(const Ctx& c, const DevMpoSite& W, int Ml1, int Ml2, int D, int d, int Mr2,
                      const cplx* Lenv, const cplx* ket, cplx* Y, const int* skip) {
  const long long per = (long long)Ml1 * D * Mr2;
  CK(zgemm(W.Dl * Ml1, D * Mr2, Ml2, 1, 1, ONE, mref(Lenv, Ml2, 1),
           mref(ket, (long long)D * Mr2, 1), ZERO, c.X, (long long)D * Mr2, 0, skip, c.st));
  CK(mpo_mix(W.lr, Ml1, d, Mr2, c.X, per, Y, per, skip, c.st));
}

void right_partial_f64(const Ctx& c, const DevMpoSite& W, int Ml2, int D, int d, int Mr1, int Mr2,
                       const cplx* Renv, const cplx* ket, cplx* Y, const int* skip) {
  const long long per = (long long)Ml2 * D * Mr1;
  // X[v][(y,s)][b] = sum_c ket[(y,s)][c] R[v][b][c]
  CK(zgemm(Ml2 * D, Mr1, Mr2, W.Dr, 1, ONE, mref(ket, Mr2, 1),
           mref(Renv, 1, Mr2, (long long)Mr1 * Mr2), ZERO, c.X, Mr1, per, skip, c.st));
  CK(mpo_mix(W.rl, Ml2, d, Mr1, c.X, per, Y, per, skip, c.st));
}

void env_left_f64(const Ctx& c, const DevMpoSite& W, int Ml1, int Mr1, int Ml2, int Mr2, int D,
                  int d, const cplx* Lenv, const cplx* bra, const cplx* ket, cplx* Lout) {
  left_partial_f64(c, W, Ml1, Ml2, D, d, Mr2, Lenv, ket, c.Y, nullptr);
  const long long per = (long long)Ml1 * D * Mr2;
  // Lout[v][b][c] = sum_{(a,s)} conj(bra[(a,s)][b]) Y[v][(a,s)][c]
  CK(zgemm(Mr1, Mr2, Ml1 * D, W.Dr, 1, ONE, mref(bra, 1, Mr1, 0, 0, 1), mref(c.Y, Mr2, 1, per),
           ZERO, Lout, Mr2, (long long)Mr1 * Mr2, nullptr, c.st));
}

void env_right_f64(const Ctx& c, const DevMpoSite& W, int Ml1, int Mr1, int Ml2, int Mr2, int D,
                   int d, const cplx* Renv, const cplx* bra, const cplx* ket, cplx* Rout) {
  right_partial_f64(c, W, Ml2, D, d, Mr1, Mr2, Renv, ket, c.Y, nullptr);
  const long long per = (long long)Ml2 * D * Mr1;
  // Rout[w][a][y] = sum_{(s,b)} conj(bra[a][(s,b)]) Y[w][y][(s,b)]
  CK(zgemm(Ml1, Ml2, D * Mr1, W.Dl, 1, ONE, mref(bra, (long long)D * Mr1, 1, 0, 0, 1),
           mref(c.Y, 1, (long long)D * Mr1, per), ZERO, Rout, Ml2, (long long)Ml1 * Ml2,
           nullptr, c.st));
}

void bond_f64(const Ctx& c, int M, int Dw, const cplx* Lenv, const cplx* Renv, const cplx* in,
              cplx* out, const int* skip) {
  const long long mm = (long long)M * M;
  CK(zgemm(Dw * M, M, M, 1, 1, ONE, mref(Lenv, M, 1), mref(in, M, 1), ZERO, c.X, M, 0, skip,
           c.st));
  CK(zgemm(M, M, M, 1, Dw, ONE, mref(c.X, M, 1, 0, mm), mref(Renv, 1, M, 0, mm), ZERO, out, M,
           0, skip, c.st));
}

// ------------------------------------------------------------------------------------
// mixed-precision H_eff on the tensor cores
// ------------------------------------------------------------------------------------
namespace {
long long r4(long long x) { return (x + 3) & ~3LL; }
}

long long heff_tc_floats(int Ml, int Mr, int D, int Dl, int Dr) {
  return 4 * r4((long long)Dl * Ml * pad4(Ml)) + 4 * r4((long long)Dr * Mr * pad4(Mr)) +
         4 * r4((long long)D * Mr * pad4(Ml)) + 2 * r4((long long)Dl * Ml * D * Mr) +
         4 * r4((long long)Dr * Ml * D * pad4(Mr)) + 64;
}

TcWork heff_tc_carve(float* base, int Ml, int Mr, int D, int Dl, int Dr, int* status) {
  TcWork w;
  float* p = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(base) + 15) & ~(uintptr_t)15);
  w.Lp = p;
  p += 4 * r4((long long)Dl * Ml * pad4(Ml));
  w.Rp = p;
  p += 4 * r4((long long)Dr * Mr * pad4(Mr));
  w.Bt = p;
  p += 4 * r4((long long)D * Mr * pad4(Ml));
  w.X = p;
  p += 2 * r4((long long)Dl * Ml * D * Mr);
  w.Yp = p;
  w.status = status;
  return w;
}

void heff_tc_envs(cudaStream_t st, const TcWork& w, int Ml, int Mr, int Dl, int Dr,
                  const cplx* Lenv, const cplx* Renv) {
  TcOperand Lp{w.Lp, Dl * Ml, Ml, pad4(Ml), 1};
  TcOperand Rp{w.Rp, Mr, Mr, pad4(Mr), Dr};
  CK(split_f64(Lenv, 0, Ml, 1, 0, Lp, st));
  CK(split_f64(Renv, (long long)Mr * Mr, Mr, 1, 0, Rp, st));
}

void heff_tc(cudaStream_t st, const TcWork& w, const DevMpoSite& W, int Ml, int Mr, int D, int d,
             const cplx* in, cplx* out) {
  const int Dl = W.Dl, Dr = W.Dr;
  TcOperand Lp{w.Lp, Dl * Ml, Ml, pad4(Ml), 1};
  TcOperand Rp{w.Rp, Mr, Mr, pad4(Mr), Dr};
  TcOperand Bt{w.Bt, D * Mr, Ml, pad4(Ml), 1};
  TcOperand Yp{w.Yp, Ml * D, Mr, pad4(Mr), Dr};
  const long long xplane = (long long)Dl * Ml * D * Mr;
  // B operand of the first contraction: in^T (rows (s,b), K = a')
  CK(split_f64_t(in, 0, (long long)D * Mr, 0, Bt, st));
  // X[(w,a)][(s,b)] = sum_y L[w,a,y] in[y,(s,b)]   -> FP32 planar
  TcGemm g1{};
  g1.M = Dl * Ml; g1.N = D * Mr; g1.K = Ml; g1.nred = 1; g1.nbatch = 1;
  g1.out_mode = 1; g1.C = w.X; g1.ldc = (long long)D * Mr; g1.sbc = 0; g1.plane = xplane;
  g1.status = w.status;
  CK(tc_gemm(Lp, Bt, g1, st));
  // Y[v][(a,s)][b] = sum W X  -> split planes
  CK(mix_split(W.lr, Ml, d, Mr, w.X, (long long)Ml * D * Mr, xplane, Yp, 0, st));
  // out[(a,s)][b] = sum_{v,c} Y[v][(a,s)][c] R[v][b][c]   -> FP64
  TcGemm g2{};
  g2.M = Ml * D; g2.N = Mr; g2.K = Mr; g2.nred = Dr; g2.nbatch = 1; g2.a_red = 1; g2.b_red = 1;
  g2.out_mode = 0; g2.C = out; g2.ldc = Mr; g2.sbc = 0; g2.status = w.status;
  CK(tc_gemm(Yp, Rp, g2, st));
}

// building blocks with engine-owned buffers
void heff_tc_prepare(cudaStream_t st, const TcBufs& b, int Ml, int Mr, int Dl, int Dr,
                     const cplx* Lenv, const cplx* Renv) {
  TcOperand Lp{b.envA, Dl * Ml, Ml, pad4(Ml), 1};
  TcOperand Rp{b.envB, Mr, Mr, pad4(Mr), Dr};
  CK(split_f64(Lenv, 0, Ml, 1, 0, Lp, st));
  CK(split_f64(Renv, (long long)Mr * Mr, Mr, 1, 0, Rp, st));
}

namespace {
// X[(w,a)][(s,c)] = sum_y L[w,a,y] ket[y,(s,c)] into b.x32 (FP32 planar), L planes in b.envA
void left_x_tc(cudaStream_t st, const TcBufs& b, int Dl, int Ml1, int Ml2, int D, int Mr2,
               const cplx* ket) {
  TcOperand Lp{b.envA, Dl * Ml1, Ml2, pad4(Ml2), 1};
  TcOperand Bt{b.siteA, D * Mr2, Ml2, pad4(Ml2), 1};
  CK(split_f64_t(ket, 0, (long long)D * Mr2, 0, Bt, st));
  TcGemm g{};
  g.M = Dl * Ml1; g.N = D * Mr2; g.K = Ml2; g.nred = 1; g.nbatch = 1;
  g.out_mode = 1; g.C = b.x32; g.ldc = (long long)D * Mr2; g.sbc = 0;
  g.plane = (long long)Dl * Ml1 * D * Mr2; g.status = b.status; g.part = b.kpart; g.part_len = b.kpart_len;
  CK(tc_gemm(Lp, Bt, g, st));
}

// X[v][(y,s)][b] = sum_c ket[(y,s)][c] R[v][b][c] into b.x32, R planes in b.envB
void right_x_tc(cudaStream_t st, const TcBufs& b, int Dr, int Ml2, int D, int Mr1, int Mr2,
                const cplx* ket) {
  TcOperand Kp{b.siteA, Ml2 * D, Mr2, pad4(Mr2), 1};
  TcOperand Rp{b.envB, Mr1, Mr2, pad4(Mr2), Dr};
  CK(split_f64(ket, 0, Mr2, 1, 0, Kp, st));
  TcGemm g{};
  g.M = Ml2 * D; g.N = Mr1; g.K = Mr2; g.nred = 1; g.nbatch = Dr; g.b_bat = 1;
  g.out_mode = 1; g.C = b.x32; g.ldc = Mr1; g.sbc = (long long)Ml2 * D * Mr1;
  g.plane = (long long)Dr * Ml2 * D * Mr1; g.status = b.status; g.part = b.kpart; g.part_len = b.kpart_len;
  CK(tc_gemm(Kp, Rp, g, st));
}
}  // namespace

void heff_tc_apply(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml, int Mr, int D,
                   int d, const cplx* in, cplx* out) {
  left_x_tc(st, b, W.Dl, Ml, Ml, D, Mr, in);
  TcOperand Yp{b.mix, Ml * D, Mr, pad4(Mr), W.Dr};
  CK(mix_split(W.lr, Ml, d, Mr, b.x32, (long long)Ml * D * Mr, (long long)W.Dl * Ml * D * Mr, Yp, 0,
               st));
  TcOperand Rp{b.envB, Mr, Mr, pad4(Mr), W.Dr};
  TcGemm g{};
  g.M = Ml * D; g.N = Mr; g.K = Mr; g.nred = W.Dr; g.nbatch = 1; g.a_red = 1; g.b_red = 1;
  g.out_mode = 0; g.C = out; g.ldc = Mr; g.status = b.status; g.part = b.kpart; g.part_len = b.kpart_len;
  CK(tc_gemm(Yp, Rp, g, st));
}

void left_partial_tc(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml1, int Ml2, int D,
                     int d, int Mr2, const cplx* Lenv, const cplx* ket, cplx* Yout) {
  TcOperand Lp{b.envA, W.Dl * Ml1, Ml2, pad4(Ml2), 1};
  CK(split_f64(Lenv, 0, Ml2, 1, 0, Lp, st));
  left_x_tc(st, b, W.Dl, Ml1, Ml2, D, Mr2, ket);
  TcOperand Yp{b.mix, Ml1 * D, Mr2, pad4(Mr2), W.Dr};
  CK(mix_split(W.lr, Ml1, d, Mr2, b.x32, (long long)Ml1 * D * Mr2,
               (long long)W.Dl * Ml1 * D * Mr2, Yp, 0, st));
  CK(planes_to_f64(Yp, Yout, st));
}

void right_partial_tc(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml2, int D, int d,
                      int Mr1, int Mr2, const cplx* Renv, const cplx* ket, cplx* Yout) {
  TcOperand Rp{b.envB, Mr1, Mr2, pad4(Mr2), W.Dr};
  CK(split_f64(Renv, (long long)Mr1 * Mr2, Mr2, 1, 0, Rp, st));
  right_x_tc(st, b, W.Dr, Ml2, D, Mr1, Mr2, ket);
  TcOperand Yp{b.mix, Ml2, D * Mr1, pad4(D * Mr1), W.Dl};
  CK(mix_split(W.rl, Ml2, d, Mr1, b.x32, (long long)Ml2 * D * Mr1,
               (long long)W.Dr * Ml2 * D * Mr1, Yp, 2, st));
  CK(planes_to_f64(Yp, Yout, st));
}

void env_left_tc(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml1, int Mr1, int Ml2,
                 int Mr2, int D, int d, const cplx* Lenv, const cplx* bra, const cplx* ket,
                 cplx* Lout) {
  TcOperand Lp{b.envA, W.Dl * Ml1, Ml2, pad4(Ml2), 1};
  CK(split_f64(Lenv, 0, Ml2, 1, 0, Lp, st));
  left_x_tc(st, b, W.Dl, Ml1, Ml2, D, Mr2, ket);
  // Y^T[v][c][(a,s)]
  TcOperand Yt{b.mix, Mr2, Ml1 * D, pad4(Ml1 * D), W.Dr};
  CK(mix_split(W.lr, Ml1, d, Mr2, b.x32, (long long)Ml1 * D * Mr2,
               (long long)W.Dl * Ml1 * D * Mr2, Yt, 1, st));
  // bra^T[b][(a,s)]
  TcOperand Bt{b.siteB, Mr1, Ml1 * D, pad4(Ml1 * D), 1};
  CK(split_f64_t(bra, 0, Mr1, 0, Bt, st));
  TcGemm g{};
  g.M = Mr1; g.N = Mr2; g.K = Ml1 * D; g.nred = 1; g.nbatch = W.Dr; g.b_bat = 1; g.conjA = 1;
  g.out_mode = 0; g.C = Lout; g.ldc = Mr2; g.sbc = (long long)Mr1 * Mr2; g.status = b.status; g.part = b.kpart; g.part_len = b.kpart_len;
  CK(tc_gemm(Bt, Yt, g, st));
}

void env_right_tc(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml1, int Mr1, int Ml2,
                  int Mr2, int D, int d, const cplx* Renv, const cplx* bra, const cplx* ket,
                  cplx* Rout) {
  TcOperand Rp{b.envB, Mr1, Mr2, pad4(Mr2), W.Dr};
  CK(split_f64(Renv, (long long)Mr1 * Mr2, Mr2, 1, 0, Rp, st));
  right_x_tc(st, b, W.Dr, Ml2, D, Mr1, Mr2, ket);
  // Y[w][y][(s,b)]
  TcOperand Yp{b.mix, Ml2, D * Mr1, pad4(D * Mr1), W.Dl};
  CK(mix_split(W.rl, Ml2, d, Mr1, b.x32, (long long)Ml2 * D * Mr1,
               (long long)W.Dr * Ml2 * D * Mr1, Yp, 2, st));
  TcOperand Bp{b.siteB, Ml1, D * Mr1, pad4(D * Mr1), 1};
  CK(split_f64(bra, 0, (long long)D * Mr1, 1, 0, Bp, st));
  TcGemm g{};
  g.M = Ml1; g.N = Ml2; g.K = D * Mr1; g.nred = 1; g.nbatch = W.Dl; g.b_bat = 1; g.conjA = 1;
  g.out_mode = 0; g.C = Rout; g.ldc = Ml2; g.sbc = (long long)Ml1 * Ml2; g.status = b.status; g.part = b.kpart; g.part_len = b.kpart_len;
  CK(tc_gemm(Bp, Yp, g, st));
}

void bond_tc_prepare(cudaStream_t st, const TcBufs& b, int M, int Dw, const cplx* Lenv,
                     const cplx* Renv) {
  TcOperand Lp{b.envA, Dw * M, M, pad4(M), 1};
  TcOperand Rp{b.envB, M, M, pad4(M), Dw};
  CK(split_f64(Lenv, 0, M, 1, 0, Lp, st));
  CK(split_f64(Renv, (long long)M * M, M, 1, 0, Rp, st));
}

void bond_tc_apply(cudaStream_t st, const TcBufs& b, int M, int Dw, const cplx* in, cplx* out) {
  TcOperand Lp{b.envA, Dw * M, M, pad4(M), 1};
  TcOperand Rp{b.envB, M, M, pad4(M), Dw};
  TcOperand Ct{b.siteA, M, M, pad4(M), 1};
  CK(split_f64_t(in, 0, M, 0, Ct, st));
  TcOperand Xp{b.mix, M, M, pad4(M), Dw};
  TcGemm g1{};
  g1.M = Dw * M; g1.N = M; g1.K = M; g1.nred = 1; g1.nbatch = 1;
  g1.out_mode = 2; g1.C = b.mix; g1.ldc = pad4(M); g1.plane = Xp.plane(); g1.status = b.status; g1.part = b.kpart; g1.part_len = b.kpart_len;
  CK(tc_gemm(Lp, Ct, g1, st));
  TcGemm g2{};
  g2.M = M; g2.N = M; g2.K = M; g2.nred = Dw; g2.nbatch = 1; g2.a_red = 1; g2.b_red = 1;
  g2.out_mode = 0; g2.C = out; g2.ldc = M; g2.status = b.status; g2.part = b.kpart; g2.part_len = b.kpart_len;
  CK(tc_gemm(Xp, Rp, g2, st));
}

// ------------------------------------------------------------------------------------
// MPO upload
// ------------------------------------------------------------------------------------
void Engine::upload_mpo(const std::vector<MpoSite>& W, DevMpo& out) {
  free_mpo(out);
  out.s.resize(W.size());
  out.maxD = 1;
  for (size_t k = 0; k < W.size(); ++k) {
    const MpoSite& h = W[k];
    DevMpoSite& s = out.s[k];
    s.Dl = h.Dl;
    s.Dr = h.Dr;
    s.d = h.d;
    s.nblk = (int)h.blocks.size();
    s.host = h.blocks;
    out.maxD = std::max(out.maxD, std::max(h.Dl, h.Dr));
    const int nb = s.nblk, d = h.d;
    // host staging: lr tables then rl tables
    std::vector<int> ilr_start(h.Dr + 1, 0), ilr_chan(nb), irl_start(h.Dl + 1, 0), irl_chan(nb);
    std::vector<cplx> olr((size_t)nb * d * d), orl((size_t)nb * d * d);
    {
      int pos = 0;
      for (int wo = 0; wo < h.Dr; ++wo) {
        ilr_start[wo] = pos;
        for (const auto& b : h.blocks)
          if (b.wr == wo) {
            ilr_chan[pos] = b.wl;
            for (int e = 0; e < d * d; ++e) olr[(size_t)pos * d * d + e] = {b.op[e].real(), b.op[e].imag()};
            ++pos;
          }
      }
      ilr_start[h.Dr] = pos;
      pos = 0;
      for (int wo = 0; wo < h.Dl; ++wo) {
        irl_start[wo] = pos;
        for (const auto& b : h.blocks)
          if (b.wl == wo) {
            irl_chan[pos] = b.wr;
            for (int e = 0; e < d * d; ++e) orl[(size_t)pos * d * d + e] = {b.op[e].real(), b.op[e].imag()};
            ++pos;
          }
      }
      irl_start[h.Dl] = pos;
    }
    const size_t ops_bytes = sizeof(cplx) * (size_t)nb * d * d;
    const size_t ops32_bytes = sizeof(float2) * (size_t)nb * d * d;
    const size_t int_bytes = sizeof(int) * (size_t)(h.Dr + 1 + nb + h.Dl + 1 + nb);
    const size_t total = 2 * ops_bytes + 2 * ops32_bytes + int_bytes + 64;
    char* mem = nullptr;
    CK(cudaMalloc(&mem, total));
    s.mem = mem;
    cplx* d_olr = reinterpret_cast<cplx*>(mem);
    cplx* d_orl = d_olr + (size_t)nb * d * d;
    float2* d_flr = reinterpret_cast<float2*>(d_orl + (size_t)nb * d * d);
    float2* d_frl = d_flr + (size_t)nb * d * d;
    int* ip = reinterpret_cast<int*>(d_frl + (size_t)nb * d * d);
    int* d_lrs = ip;
    int* d_lrc = d_lrs + h.Dr + 1;
    int* d_rls = d_lrc + nb;
    int* d_rlc = d_rls + h.Dl + 1;
    std::vector<float2> flr(olr.size()), frl(orl.size());
    for (size_t e = 0; e < olr.size(); ++e) flr[e] = make_float2((float)olr[e].x, (float)olr[e].y);
    for (size_t e = 0; e < orl.size(); ++e) frl[e] = make_float2((float)orl[e].x, (float)orl[e].y);
    if (nb > 0) {
      CK(cudaMemcpy(d_flr, flr.data(), ops32_bytes, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_frl, frl.data(), ops32_bytes, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_olr, olr.data(), ops_bytes, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_orl, orl.data(), ops_bytes, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_lrc, ilr_chan.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_rlc, irl_chan.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(d_lrs, ilr_start.data(), sizeof(int) * (h.Dr + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_rls, irl_start.data(), sizeof(int) * (h.Dl + 1), cudaMemcpyHostToDevice));
    s.lr = MixTable{h.Dr, d_lrs, d_lrc, d_olr, d_flr, nb};
    s.rl = MixTable{h.Dl, d_rls, d_rlc, d_orl, d_frl, nb};
  }
}

void Engine::free_mpo(DevMpo& m) {
  for (auto& s : m.s)
    if (s.mem) cudaFree(s.mem);
  m.s.clear();
}

// ------------------------------------------------------------------------------------
// construction / workspace
// ------------------------------------------------------------------------------------
Engine::Engine(const ModelParams& p) : P(p) {
  CK(cudaGetDevice(&dev_));
  sites_ = chain_sites(P);
  rebuild_mpos();
  CK(cudaMalloc(&status_, sizeof(int) * 4));
  CK(cudaMemset(status_, 0, sizeof(int) * 4));
  bs_.noconv = status_ + 3;
  CK(cudaMalloc(&lz_, sizeof(LzState)));
  CK(cudaMalloc(&scal_, sizeof(double) * 8));
  CK(cudaMalloc(&part_d_, sizeof(double) * NBLK));
  CK(cudaMalloc(&red_cnt_, sizeof(unsigned) * (KMAX + 2)));
  CK(cudaMemset(red_cnt_, 0, sizeof(unsigned) * (KMAX + 2)));
  CK(cudaMallocHost(&h_pinned_, sizeof(int) * 8));
  CK(cudaMallocHost(&h_pinned_d_, sizeof(double) * 4));
  for (auto& e : ev_) CK(cudaEventCreate(&e));
  for (auto& e : qr_ev_) CK(cudaEventCreate(&e));
  for (auto& e : lz_ev_) CK(cudaEventCreate(&e));
}

Engine::~Engine() {
  clear_graphs();
  if (own_stream_) {
    cudaStreamSynchronize(own_stream_);
    cudaStreamDestroy(own_stream_);
  }
  free_mps(psi_b_);
  free_mps(psi1_);
  free_mps(psi2_);
  free_mpo(H_);
  free_mpo(J_);
  free_mpo(I_);
  cplx* bufs[] = {X_, Y_, V_, Kout_, T1_, Cb_, Rb_, Ex_, env_tmp_[0], env_tmp_[1]};
  for (cplx* b : bufs)
    if (b) cudaFree(b);
  if (part_d_) cudaFree(part_d_);
  if (red_cnt_) cudaFree(red_cnt_);
  if (scal_) cudaFree(scal_);
  if (lz_) cudaFree(lz_);
  if (status_) cudaFree(status_);
  if (qr_.part) cudaFree(qr_.part);
  if (qr_.partn) cudaFree(qr_.partn);
  if (qr_.bar) cudaFree(qr_.bar);
  if (qb_scratch_) cudaFree(qb_scratch_);
  if (qb_acc_) cudaFree(qb_acc_);
  if (h_pinned_) cudaFreeHost(h_pinned_);
  if (h_pinned_d_) cudaFreeHost(h_pinned_d_);
  for (auto& e : ev_)
    if (e) cudaEventDestroy(e);
  for (auto& e : qr_ev_)
    if (e) cudaEventDestroy(e);
  for (auto& e : lz_ev_)
    if (e) cudaEventDestroy(e);
  for (float* p : {tcb_.envA, tcb_.envB, tcb_.siteA, tcb_.siteB, tcb_.x32, tcb_.mix, tcb_.kpart})
    if (p) cudaFree(p);
  for (void* p : {(void*)bs_.W, (void*)bs_.T, (void*)bs_.P, (void*)bs_.part, (void*)bs_.partn,
                  (void*)bs_.bar, (void*)bs_.mv})
    if (p) cudaFree(p);
  if (h_mv_) cudaFreeHost(h_mv_);
}

void Engine::rebuild_mpos() {
  twin_.reset();     // built from the old parameters; made again at the next realtime_init
  twin_on_ = false;
  sites_ = chain_sites(P);
  upload_mpo(hamiltonian_mpo(P), H_);
  upload_mpo(current_mpo(P), J_);
  upload_mpo(identity_mpo(P), I_);
  prepared_ = false;
  rt_ready_ = false;
}

void Engine::set_precision(int p) {
  if (p != TDMRG_PREC_C128 && p != TDMRG_PREC_C64_3XTF32)
    throw Failure{TDMRG_ERR_ARG, "unknown precision"};
  if (p != precision_) {
    clear_graphs();
    precision_ = p;
    if (!ktol_user_) ktol_ = (p == TDMRG_PREC_C128) ? 1e-13 : 1e-7;
    if (!rank_tol_user_) rank_tol_ = (p == TDMRG_PREC_C128) ? 1e-12 : kMixedRankTol;
    prepared_ = false;
    rt_ready_ = false;
  }
}

void Engine::set_krylov(double tol, int kmax, int fixed_k) {
  if (!(tol > 0.0) || kmax < 1 || kmax > KMAX || fixed_k < 0 || fixed_k > KMAX)
    throw Failure{TDMRG_ERR_ARG, "krylov: need tol > 0, 1 <= kmax <= 32, 0 <= fixed_k <= 32"};
  if (graphs_ && fixed_k <= 0)
    throw Failure{TDMRG_ERR_ARG, "graph mode needs a fixed Krylov dimension"};
  clear_graphs();
  ktol_ = tol;
  ktol_user_ = true;
  kmax_ = kmax;
  fixed_k_ = fixed_k;
}

void Engine::ensure_workspace(long long maxsite, long long maxxy, int maxbond, int maxm) {
  if (maxsite > ws_site_) {
    for (cplx** b : {&V_, &Kout_, &T1_}) {
      if (*b) cudaFree(*b);
      *b = nullptr;
    }
    CK(cudaMalloc(&V_, sizeof(cplx) * (size_t)(KMAX + 1) * maxsite));
    CK(cudaMalloc(&Kout_, sizeof(cplx) * (size_t)maxsite));
    CK(cudaMalloc(&T1_, sizeof(cplx) * (size_t)maxsite));
    ws_site_ = maxsite;
  }
  if (maxxy > ws_xy_) {
    for (cplx** b : {&X_, &Y_}) {
      if (*b) cudaFree(*b);
      *b = nullptr;
    }
    CK(cudaMalloc(&X_, sizeof(cplx) * (size_t)maxxy));
    CK(cudaMalloc(&Y_, sizeof(cplx) * (size_t)maxxy));
    ws_xy_ = maxxy;
  }
  if (maxbond > ws_bond_) {
    for (cplx** b : {&Cb_, &Rb_}) {
      if (*b) cudaFree(*b);
      *b = nullptr;
    }
    CK(cudaMalloc(&Cb_, sizeof(cplx) * (size_t)maxbond * maxbond));
    CK(cudaMalloc(&Rb_, sizeof(cplx) * (size_t)maxbond * maxbond));
    ws_bond_ = maxbond;
  }
  ensure_bond_scratch(maxbond);
  if (maxm > ws_m_) {
    if (qr_.part) cudaFree(qr_.part);
    if (qr_.partn) cudaFree(qr_.partn);
    if (qr_.bar) cudaFree(qr_.bar);
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    qr_.gmax = sms;
    qr_.nmax = maxm;
    CK(cudaMalloc(&qr_.part, sizeof(cplx) * 2 * (size_t)sms * (maxm + 1)));
    CK(cudaMalloc(&qr_.partn, sizeof(double) * 2 * (size_t)sms));
    CK(cudaMalloc(&qr_.bar, sizeof(unsigned) * 2));
    if (qb_scratch_) cudaFree(qb_scratch_);
    if (qb_acc_) cudaFree(qb_acc_);
    qb_len_ = gauge_qr_blocked_scratch(maxm, sms);
    CK(cudaMalloc(&qb_scratch_, sizeof(cplx) * (size_t)qb_len_));
    CK(cudaMalloc(&qb_acc_, (size_t)maxm + 16));
    ws_m_ = maxm;
  }
}

long long Engine::env_size(const DevMps& s, int k, int Dw, bool left) const {
  const long long M = left ? s.Mb[k] : s.Mb[k + 1];
  return (long long)Dw * M * M;
}

void Engine::alloc_mps(DevMps& s, int M) {
  clear_graphs();
  free_mps(s);
  const int L = (int)sites_.size();
  s.Mb = bond_dimensions(sites_, M);
  s.D.resize(L);
  s.d.resize(L);
  s.A.assign(L, nullptr);
  s.Lenv.assign(L, nullptr);
  s.Renv.assign(L, nullptr);
  for (int k = 0; k < L; ++k) {
    s.d[k] = sites_[k].d;
    s.D[k] = sites_[k].d * sites_[k].d;
    CK(cudaMalloc(&s.A[k], sizeof(cplx) * (size_t)s.size(k)));
    CK(cudaMalloc(&s.Lenv[k], sizeof(cplx) * (size_t)env_size(s, k, H_.s[k].Dl, true)));
    CK(cudaMalloc(&s.Renv[k], sizeof(cplx) * (size_t)env_size(s, k, H_.s[k].Dr, false)));
  }
  long long maxsite = 1, maxxy = 1, maxenv = 1;
  int maxbond = 1;
  const int Dmax = std::max(H_.maxD, J_.maxD);
  for (int k = 0; k < L; ++k) {
    maxsite = std::max(maxsite, s.size(k));
    maxxy = std::max(maxxy, (long long)Dmax * s.size(k));
    maxbond = std::max(maxbond, s.Mb[k + 1]);
    maxenv = std::max(maxenv, env_size(s, k, Dmax, true));
    maxenv = std::max(maxenv, env_size(s, k, Dmax, false));
  }
  maxxy = std::max(maxxy, (long long)Dmax * maxbond * maxbond);
  ensure_workspace(maxsite, maxxy, maxbond, maxbond);
  if (mixed()) alloc_tc(s);
  if (maxenv > env_tmp_size_) {
    for (int i = 0; i < 2; ++i) {
      if (env_tmp_[i]) cudaFree(env_tmp_[i]);
      CK(cudaMalloc(&env_tmp_[i], sizeof(cplx) * (size_t)maxenv));
    }
    env_tmp_size_ = maxenv;
  }
}

void Engine::alloc_tc(const DevMps& s) {
  const int Dmax = std::max(H_.maxD, J_.maxD);
  long long site = 1, env = 1, x = 1;
  for (int k = 0; k < s.L(); ++k) {
    const long long Ml = s.Mb[k], Mr = s.Mb[k + 1], D = s.D[k];
    const long long cands[4] = {D * Mr * pad4((int)Ml), Ml * D * pad4((int)Mr),
                                Mr * pad4((int)(Ml * D)), Ml * pad4((int)(D * Mr))};
    for (long long c : cands) site = std::max(site, c);
    env = std::max(env, (long long)Dmax * Ml * pad4((int)Ml));
    env = std::max(env, (long long)Dmax * Mr * pad4((int)Mr));
    x = std::max(x, (long long)Dmax * Ml * D * Mr);
  }
  if (site > tc_site_ || env > tc_env_ || x > tc_x_) {
    for (float** p : {&tcb_.envA, &tcb_.envB, &tcb_.siteA, &tcb_.siteB, &tcb_.x32, &tcb_.mix}) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
    CK(cudaMalloc(&tcb_.envA, sizeof(float) * 4 * env));
    CK(cudaMalloc(&tcb_.envB, sizeof(float) * 4 * env));
    CK(cudaMalloc(&tcb_.siteA, sizeof(float) * 4 * site));
    CK(cudaMalloc(&tcb_.siteB, sizeof(float) * 4 * site));
    CK(cudaMalloc(&tcb_.x32, sizeof(float) * 2 * x));
    CK(cudaMalloc(&tcb_.mix, sizeof(float) * 4 * (long long)Dmax * site));
    if (!tcb_.kpart) {
      tcb_.kpart_len = 4LL << 20;
      CK(cudaMalloc(&tcb_.kpart, sizeof(float) * tcb_.kpart_len));
    }
    tc_site_ = site;
    tc_env_ = env;
    tc_x_ = x;
  }
  tcb_.status = status_ + 2;
}

void Engine::env_left_any(const DevMpoSite& W, int Ml1, int Mr1, int Ml2, int Mr2, int D, int d,
                          const cplx* Lenv, const cplx* bra, const cplx* ket, cplx* Lout) {
  if (mixed())
    env_left_tc(st_, tcb_, W, Ml1, Mr1, Ml2, Mr2, D, d, Lenv, bra, ket, Lout);
  else
    env_left_f64(ctx(), W, Ml1, Mr1, Ml2, Mr2, D, d, Lenv, bra, ket, Lout);
}

void Engine::env_right_any(const DevMpoSite& W, int Ml1, int Mr1, int Ml2, int Mr2, int D, int d,
                           const cplx* Renv, const cplx* bra, const cplx* ket, cplx* Rout) {
  if (mixed())
    env_right_tc(st_, tcb_, W, Ml1, Mr1, Ml2, Mr2, D, d, Renv, bra, ket, Rout);
  else
    env_right_f64(ctx(), W, Ml1, Mr1, Ml2, Mr2, D, d, Renv, bra, ket, Rout);
}

void Engine::free_mps(DevMps& s) {
  for (auto* p : s.A)
    if (p) cudaFree(p);
  for (auto* p : s.Lenv)
    if (p) cudaFree(p);
  for (auto* p : s.Renv)
    if (p) cudaFree(p);
  s.A.clear();
  s.Lenv.clear();
  s.Renv.clear();
}

void Engine::copy_mps(const DevMps& src, DevMps& dst) {
  if (dst.A.size() != src.A.size() || dst.Mb != src.Mb) {
    clear_graphs();
    free_mps(dst);
    dst.Mb = src.Mb;
    dst.D = src.D;
    dst.d = src.d;
    const int L = src.L();
    dst.A.assign(L, nullptr);
    dst.Lenv.assign(L, nullptr);
    dst.Renv.assign(L, nullptr);
    for (int k = 0; k < L; ++k) {
      CK(cudaMalloc(&dst.A[k], sizeof(cplx) * (size_t)src.size(k)));
      CK(cudaMalloc(&dst.Lenv[k], sizeof(cplx) * (size_t)env_size(src, k, H_.s[k].Dl, true)));
      CK(cudaMalloc(&dst.Renv[k], sizeof(cplx) * (size_t)env_size(src, k, H_.s[k].Dr, false)));
    }
  }
  for (int k = 0; k < src.L(); ++k)
    CK(cudaMemcpyAsync(dst.A[k], src.A[k], sizeof(cplx) * (size_t)src.size(k),
                       cudaMemcpyDeviceToDevice, st_));
}

double Engine::tic() {
  if (!prof_ || capturing_) return 0.0;
  CK(cudaStreamSynchronize(st_));
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void Engine::toc(double& acc, double t0) {
  if (!prof_ || capturing_) return;
  CK(cudaStreamSynchronize(st_));
  acc += std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count() - t0;
}

void Engine::set_ones(cplx* p) {
  static const cplx one = {1.0, 0.0};
  CK(cudaMemcpyAsync(p, &one, sizeof(cplx), cudaMemcpyHostToDevice, st_));
  stats.h2d_bytes += sizeof(cplx);
}

// ------------------------------------------------------------------------------------
// numerics helpers
// ------------------------------------------------------------------------------------
double Engine::norm2_dev(const cplx* x, long long n) {
  CK(znorm2(n, x, scal_, part_d_, red_cnt_ + KMAX + 1, nullptr, st_));
  CK(cudaMemcpyAsync(h_pinned_d_, scal_, sizeof(double), cudaMemcpyDeviceToHost, st_));
  CK(cudaStreamSynchronize(st_));
  stats.d2h_bytes += sizeof(double);
  return h_pinned_d_[0];
}

void Engine::scale_dev(cplx* x, long long n, double f) {
  h_pinned_d_[1] = f;
  CK(cudaMemcpyAsync(scal_ + 1, h_pinned_d_ + 1, sizeof(double), cudaMemcpyHostToDevice, st_));
  stats.h2d_bytes += sizeof(double);
  CK(zscale_by(n, x, scal_ + 1, nullptr, st_));
  CK(cudaStreamSynchronize(st_));
}

void Engine::ensure_bond_scratch(int maxbond) {
  const long long maxn = (long long)maxbond * maxbond;
  const int maxDw = std::max(H_.maxD, J_.maxD);
  if (maxn <= bs_.maxn && maxDw <= bs_.maxDw) return;
  for (void* p : {(void*)bs_.W, (void*)bs_.T, (void*)bs_.P})
    if (p) cudaFree(p);
  bs_.W = nullptr;
  bs_.T = bs_.P = nullptr;
  CK(cudaMalloc(&bs_.W, sizeof(cplx) * (size_t)maxn));
  CK(cudaMalloc(&bs_.T, sizeof(float2) * (size_t)maxDw * maxn));
  CK(cudaMalloc(&bs_.P, sizeof(float2) * (size_t)maxDw * maxn));
  if (!bs_.part) {
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    bs_.gmax = sms;
    CK(cudaMalloc(&bs_.part, sizeof(cplx) * 2 * (size_t)sms * (KMAX + 1)));
    CK(cudaMalloc(&bs_.partn, sizeof(double) * 2 * (size_t)sms));   // 2 * gmax: lz_step
    CK(cudaMalloc(&bs_.bar, sizeof(unsigned) * 2));
    CK(cudaMalloc(&bs_.mv, sizeof(unsigned long long)));
    CK(cudaMemset(bs_.mv, 0, sizeof(unsigned long long)));
    CK(cudaMallocHost(&h_mv_, sizeof(unsigned long long)));
    mv_seen_ = 0;
  }
  bs_.maxn = maxn;
  bs_.maxDw = maxDw;
}

// exp(tau K) Cb_ -> Rb_ in one cooperative launch (mixed path); the number of Krylov vectors
// it used is accumulated on the device and collected by check_status().
void Engine::bond_exp(int M, int Dw, const cplx* Le, const cplx* Re, double tr, double ti) {
  const int cap0 = fixed_k_ > 0 ? fixed_k_ : kmax_;
  const int kcap = (int)std::min<long long>(cap0, (long long)M * M);
  CK(bond_exp_fused(M, Dw, Le, Re, Cb_, Rb_, V_, bs_, status_ + 1, tr, ti, ktol_, kcap,
                    fixed_k_ > 0 ? 1 : 0, qr_gcap_, st_));
}

void Engine::check_status() {
  CK(cudaMemcpyAsync(h_pinned_ + 1, status_, 3 * sizeof(int), cudaMemcpyDeviceToHost, st_));
  CK(cudaMemcpyAsync(h_pinned_ + 7, status_ + 3, sizeof(int), cudaMemcpyDeviceToHost, st_));
  stats.d2h_bytes += 4 * sizeof(int);
  if (bs_.mv) {
    CK(cudaMemcpyAsync(h_mv_, bs_.mv, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st_));
    stats.d2h_bytes += sizeof(unsigned long long);
  }
  CK(cudaStreamSynchronize(st_));
  harvest_qr_events();
  if (bs_.mv) {
    const double used = (double)(*h_mv_ - mv_seen_);
    mv_seen_ = *h_mv_;
    stats.bond_matvecs += used;
    stats.krylov_vectors += used;
  }
  const int qr = h_pinned_[1], lz = h_pinned_[2], tc = h_pinned_[3], nc = h_pinned_[7];
  if (qr || lz || tc || nc) {
    // the state of this step is not usable, but the handle is: clear the words so that the
    // next call (a new preparation) starts from a clean status
    CK(cudaMemsetAsync(status_, 0, 4 * sizeof(int), st_));
    CK(cudaStreamSynchronize(st_));
  }
  if (qr == 1) throw Failure{TDMRG_ERR_TIMEOUT, "gauge QR grid barrier timed out"};
  if (lz == 1) throw Failure{TDMRG_ERR_TIMEOUT, "Lanczos grid barrier timed out"};
  if (qr == 2) throw Failure{TDMRG_ERR_CUDA, "gauge QR ran out of completion vectors"};
  if (tc != 0) throw Failure{TDMRG_ERR_TIMEOUT, "tensor-core pipeline wait timed out"};
  if (nc != 0)
    throw Failure{TDMRG_ERR_NOCONV,
                  "a Krylov exponential stopped at kmax with its error estimate above 1e3 tol"};
}

// Every gauge QR outside a graph capture is bracketed by a pair of events; the pairs are read
// at the next status check (the stream is synchronised there) or when the ring is full.
void Engine::gauge_qr_dev(int m, int n, QrRef Y, int p, QrRef E, cplx* Q, cplx* R, int* src) {
  const double t0 = tic();
  const bool timed = !capturing_;
  if (timed) {
    if (qr_ev_n_ == QR_EV) harvest_qr_events();
    CK(cudaEventRecord(qr_ev_[2 * qr_ev_n_], st_));
  }
  CK(gauge_qr_blocked(m, n, Y, p, E, Q, R, qb_scratch_, qb_len_, qb_acc_, qr_, status_, st_,
                      qr_gcap_, rank_tol_, src));
  if (timed) {
    CK(cudaEventRecord(qr_ev_[2 * qr_ev_n_ + 1], st_));
    qr_ev_bulk_[qr_ev_n_] = m >= 4096 ? 1 : 0;
    ++qr_ev_n_;
    stats.qr_flops += 8.0 * m * (double)n * n;   // one Gram-Schmidt pass
    if (m >= 4096) {
      stats.qr_bulk_flops += 8.0 * m * (double)n * n;
      stats.qr_bulk_n += 1;
    }
  }
  toc(stats.t_qr, t0);
  stats.qrs += 1;
}

// reads the event pairs of the gauge QRs and of the Lanczos steps recorded so far
void Engine::harvest_qr_events() {
  if (qr_ev_n_ > 0) {
    CK(cudaEventSynchronize(qr_ev_[2 * qr_ev_n_ - 1]));
    for (int i = 0; i < qr_ev_n_; ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, qr_ev_[2 * i], qr_ev_[2 * i + 1]));
      stats.qr_ms += ms;
      if (qr_ev_bulk_[i]) stats.qr_bulk_ms += ms;
    }
    qr_ev_n_ = 0;
  }
  if (lz_ev_n_ > 0) {
    CK(cudaEventSynchronize(lz_ev_[2 * lz_ev_n_ - 1]));
    for (int i = 0; i < lz_ev_n_; ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, lz_ev_[2 * i], lz_ev_[2 * i + 1]));
      stats.lz_ms += ms;
    }
    lz_ev_n_ = 0;
  }
}

void Engine::absorb_left(const cplx* C, int M, cplx* A, long long ncols) {
  if (mixed()) {
    // T1[b][c] = sum_b' C[b][b'] A[b'][c] on the tensor cores
    TcOperand Cp{tcb_.envA, M, M, pad4(M), 1};
    TcOperand At{tcb_.siteA, (int)ncols, M, pad4(M), 1};
    CK(split_f64(C, 0, M, 1, 0, Cp, st_));
    CK(split_f64_t(A, 0, ncols, 0, At, st_));
    TcGemm g{};
    g.M = M; g.N = (int)ncols; g.K = M; g.nred = 1; g.nbatch = 1;
    g.out_mode = 0; g.C = T1_; g.ldc = ncols; g.status = tcb_.status; g.part = tcb_.kpart; g.part_len = tcb_.kpart_len;
    CK(tc_gemm(Cp, At, g, st_));
  } else {
    CK(zgemm(M, (int)ncols, M, 1, 1, ONE, mref(C, M, 1), mref(A, ncols, 1), ZERO, T1_, ncols, 0,
             nullptr, st_));
  }
  CK(cudaMemcpyAsync(A, T1_, sizeof(cplx) * (size_t)M * ncols, cudaMemcpyDeviceToDevice, st_));
}

void Engine::absorb_right(cplx* A, long long nrows, const cplx* C, int M) {
  if (mixed()) {
    // T1[r][b] = sum_b' A[r][b'] C[b'][b] on the tensor cores
    TcOperand Ap{tcb_.siteA, (int)nrows, M, pad4(M), 1};
    TcOperand Ct{tcb_.envA, M, M, pad4(M), 1};
    CK(split_f64(A, 0, M, 1, 0, Ap, st_));
    CK(split_f64_t(C, 0, M, 0, Ct, st_));
    TcGemm g{};
    g.M = (int)nrows; g.N = M; g.K = M; g.nred = 1; g.nbatch = 1;
    g.out_mode = 0; g.C = T1_; g.ldc = M; g.status = tcb_.status; g.part = tcb_.kpart; g.part_len = tcb_.kpart_len;
    CK(tc_gemm(Ap, Ct, g, st_));
  } else {
    CK(zgemm((int)nrows, M, M, 1, 1, ONE, mref(A, M, 1), mref(C, M, 1), ZERO, T1_, M, 0, nullptr,
             st_));
  }
  CK(cudaMemcpyAsync(A, T1_, sizeof(cplx) * (size_t)M * nrows, cudaMemcpyDeviceToDevice, st_));
}

// ------------------------------------------------------------------------------------
// gauge shifts
// ------------------------------------------------------------------------------------
// center (Ml*D x Mr) = Q Cbond; Q -> A_k; L_{k+1} updated.  Completion candidates are the
// columns of the left part of H_eff applied to the center.
void Engine::shift_right(DevMps& s, int k, const cplx* center, cplx* Cbond) {
  const DevMpoSite& W = H_.s[k];
  const int Ml = s.Mb[k], Mr = s.Mb[k + 1], D = s.D[k], d = s.d[k];
  if (mixed())
    left_partial_tc(st_, tcb_, W, Ml, Ml, D, d, Mr, s.Lenv[k], center, Y_);
  else
    left_partial_f64(ctx(), W, Ml, Ml, D, d, Mr, s.Lenv[k], center, Y_, nullptr);
  gauge_qr_dev(Ml * D, Mr, qref(center, Mr, 1, NOSPLIT, 0, 0), W.Dr * Mr,
               qref(Y_, Mr, 1, Mr, (long long)Ml * D * Mr, 0), s.A[k], Cbond);
  env_left_any(W, Ml, Mr, Ml, Mr, D, d, s.Lenv[k], s.A[k], s.A[k], s.Lenv[k + 1]);
  stats.env_updates += 1;
}

// center (Ml x D*Mr) = Cbond Q; Q -> A_k; R_{k-1} updated.  Works on Y = center^H.
void Engine::shift_left(DevMps& s, int k, const cplx* center, cplx* Cbond) {
  const DevMpoSite& W = H_.s[k];
  const int Ml = s.Mb[k], Mr = s.Mb[k + 1], D = s.D[k], d = s.d[k];
  if (mixed())
    right_partial_tc(st_, tcb_, W, Ml, D, d, Mr, Mr, s.Renv[k], center, Y_);
  else
    right_partial_f64(ctx(), W, Ml, D, d, Mr, Mr, s.Renv[k], center, Y_, nullptr);
  gauge_qr_dev(D * Mr, Ml, qref(center, 1, (long long)D * Mr, NOSPLIT, 0, 1), W.Dl * Ml,
               qref(Y_, 1, (long long)D * Mr, NOSPLIT, 0, 1), T1_, Rb_);
  CK(ztranspose(D * Mr, Ml, T1_, s.A[k], 1, st_));
  CK(ztranspose(Ml, Ml, Rb_, Cbond, 1, st_));
  env_right_any(W, Ml, Mr, Ml, Mr, D, d, s.Renv[k], s.A[k], s.A[k], s.Renv[k - 1]);
  stats.env_updates += 1;
}

// The bond factors carry the norm of |I> on the one-carrier sector, which grows like the
// square root of the sector's dimension (e^138 for 32 molecules with four modes): each one is
// normalised in FP64 before it is absorbed (the tensor-core absorb holds FP32 exponents) and
// log ||.||^2 is accumulated on the device.
void Engine::right_canonicalize(DevMps& s) {
  const int L = s.L();
  set_ones(s.Lenv[0]);
  set_ones(s.Renv[L - 1]);
  for (int k = L - 1; k > 0; --k) {
    shift_left(s, k, s.A[k], Cb_);
    renormalize(Cb_, (long long)s.Mb[k] * s.Mb[k]);
    absorb_right(s.A[k - 1], (long long)s.Mb[k - 1] * s.D[k - 1], Cb_, s.Mb[k]);
  }
}

void Engine::build_right_envs(DevMps& s) {
  const int L = s.L();
  set_ones(s.Lenv[0]);
  set_ones(s.Renv[L - 1]);
  for (int k = L - 1; k > 0; --k) {
    const int Ml = s.Mb[k], Mr = s.Mb[k + 1];
    env_right_any(H_.s[k], Ml, Mr, Ml, Mr, s.D[k], s.d[k], s.Renv[k], s.A[k], s.A[k],
                  s.Renv[k - 1]);
  }
}

// ------------------------------------------------------------------------------------
// the projector-splitting step
// ------------------------------------------------------------------------------------
void Engine::site_update(DevMps& s, int k, double hr, double hi) {
  const DevMpoSite& W = H_.s[k];
  const int Ml = s.Mb[k], Mr = s.Mb[k + 1], D = s.D[k], d = s.d[k];
  const double flops = 8.0 * W.Dl * Ml * (double)Ml * D * Mr + 8.0 * W.Dr * Ml * (double)D * Mr * Mr;
  const cplx* Le = s.Lenv[k];
  const cplx* Re = s.Renv[k];
  Ctx c = ctx();
  int nev = 0;
  const bool mx = mixed();
  if (mx) heff_tc_prepare(st_, tcb_, Ml, Mr, W.Dl, W.Dr, Le, Re);
  const bool timed = !capturing_;
  const int used = krylov(s.size(k), s.A[k], Kout_, hr, hi,
                          [&](const cplx* in, cplx* out, const int* skip) {
    if (timed) CK(cudaEventRecord(ev_[2 * nev], st_));
    if (mx)
      heff_tc_apply(st_, tcb_, W, Ml, Mr, D, d, in, out);
    else
      heff_f64(c, W, Ml, Mr, D, d, Le, Re, in, out, skip);
    if (timed) CK(cudaEventRecord(ev_[2 * nev + 1], st_));
    ++nev;
  });
  stats.matvecs += used;
  stats.heff_flops += used * flops;
  if (timed && used > 0) CK(cudaEventSynchronize(ev_[2 * (used - 1) + 1]));
  for (int i = 0; timed && i < used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev_[2 * i], ev_[2 * i + 1]));
    stats.heff_ms += ms;
  }
  stats.site_updates += 1;
}

namespace {
Stats stats_diff(const Stats& a, const Stats& b) {
  Stats d;
  d.site_updates = a.site_updates - b.site_updates;
  d.matvecs = a.matvecs - b.matvecs;
  d.heff_flops = a.heff_flops - b.heff_flops;
  d.krylov_vectors = a.krylov_vectors - b.krylov_vectors;
  d.bond_matvecs = a.bond_matvecs - b.bond_matvecs;
  d.qrs = a.qrs - b.qrs;
  d.completions = a.completions - b.completions;
  d.env_updates = a.env_updates - b.env_updates;
  d.h2d_bytes = a.h2d_bytes - b.h2d_bytes;
  d.d2h_bytes = a.d2h_bytes - b.d2h_bytes;
  d.replayed_launches = a.replayed_launches - b.replayed_launches;
  return d;
}
void stats_add(Stats& a, const Stats& d) {
  a.site_updates += d.site_updates;
  a.matvecs += d.matvecs;
  a.heff_flops += d.heff_flops;
  a.krylov_vectors += d.krylov_vectors;
  a.bond_matvecs += d.bond_matvecs;
  a.qrs += d.qrs;
  a.completions += d.completions;
  a.env_updates += d.env_updates;
  a.h2d_bytes += d.h2d_bytes;
  a.d2h_bytes += d.d2h_bytes;
  a.replayed_launches += d.replayed_launches;
}
}  // namespace

void Engine::set_graphs(bool on, int qr_cap) {
  if (on && fixed_k_ <= 0)
    throw Failure{TDMRG_ERR_ARG, "graph mode needs a fixed Krylov dimension (set_krylov fixed_k)"};
  clear_graphs();
  if (on && twin_on_) {
    // graph mode steps both states on this engine: take the second state back from the twin
    CK(cudaStreamSynchronize(twin_->st_));
    for (int k = 0; k < psi2_.L(); ++k)
      CK(cudaMemcpyAsync(psi2_.A[k], twin_->psi1_.A[k], sizeof(cplx) * (size_t)psi2_.size(k),
                         cudaMemcpyDeviceToDevice, st_));
    build_right_envs(psi2_);
    CK(cudaStreamSynchronize(st_));
    twin_on_ = false;
  }
  graphs_ = on;
  qr_gcap_ = qr_cap;
  if (on && st_ == 0) {
    if (!own_stream_) CK(cudaStreamCreateWithFlags(&own_stream_, cudaStreamNonBlocking));
    st_ = own_stream_;
  }
}

void Engine::clear_graphs() {
  for (auto& g : step_graphs_)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  step_graphs_.clear();
}

const Engine::StepGraph& Engine::step_graph(DevMps& s, double tr, double ti, int half) {
  for (const auto& g : step_graphs_)
    if (g.state == &s && g.tr == tr && g.ti == ti && g.half == half) return g;
  const Stats before = stats;
  const long long launches0 = launch_count();
  capturing_ = true;
  CK(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t graph = nullptr;
  try {
    tdvp_step_body(s, tr, ti, half);
  } catch (...) {
    cudaStreamEndCapture(st_, &graph);
    if (graph) cudaGraphDestroy(graph);
    capturing_ = false;
    stats = before;
    throw;
  }
  capturing_ = false;
  CK(cudaStreamEndCapture(st_, &graph));
  StepGraph g{&s, tr, ti, half, nullptr, stats_diff(stats, before)};
  g.delta.replayed_launches = (double)(launch_count() - launches0);
  // the captured launches did not run: the counter keeps counting real launches only
  count_launch(-(int)(launch_count() - launches0));
  stats = before;
  const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
  step_graphs_.push_back(g);
  return step_graphs_.back();
}

void Engine::tdvp_step(DevMps& s, double tr, double ti) {
  if (graphs_) {
    const StepGraph& g = step_graph(s, tr, ti);
    CK(cudaGraphLaunch(g.exec, st_));
    stats_add(stats, g.delta);
    check_status();
    return;
  }
  tdvp_step_body(s, tr, ti);
  check_status();
}

void Engine::sync_and_check() { check_status(); }

Stats Engine::capture_realtime_half(double dt, int half) {
  if (!rt_ready_) throw Failure{TDMRG_ERR_STATE, "realtime half-step before realtime_init"};
  if (!graphs_) throw Failure{TDMRG_ERR_STATE, "batched stepping needs graph mode"};
  if (half != 1 && half != 2) throw Failure{TDMRG_ERR_ARG, "half-step: half must be 1 or 2"};
  const Stats before = stats;
  const long long launches0 = launch_count();
  capturing_ = true;
  try {
    tdvp_step_body(psi1_, 0.0, -dt, half);
    tdvp_step_body(psi2_, 0.0, -dt, half);
  } catch (...) {
    capturing_ = false;
    stats = before;
    throw;
  }
  capturing_ = false;
  Stats d = stats_diff(stats, before);
  d.replayed_launches = (double)(launch_count() - launches0);
  count_launch(-(int)(launch_count() - launches0));
  stats = before;
  return d;
}

void Engine::add_stats(const Stats& d) { stats_add(stats, d); }

void Engine::reset_stats() {
  harvest_qr_events();
  stats = Stats();
  stats.launches_at_reset = (double)launch_count();
  if (twin_) twin_->reset_stats();
}

// Imaginary time: the center is multiplied by exp(-tau H_eff / 2) at every site and by
// exp(+tau K / 2) at every bond, so its norm drifts by about exp(-tau <H> / 2) per half step
// and by e^(-beta <H>) over the whole preparation.  It is renormalised after each bond
// absorption, which keeps the tensor-core operands near unit scale, and log ||.||^2
// accumulates on the device into log Z (a scalar: the direction of the state is unchanged).
void Engine::renormalize(cplx* A, long long n) {
  CK(znorm2(n, A, scal_ + 2, part_d_, red_cnt_ + KMAX + 1, nullptr, st_));
  CK(znormalize_log(n, A, scal_ + 2, scal_ + 3, st_));
}

void Engine::tdvp_step_body(DevMps& s, double tr, double ti, int half) {
  const double hr = 0.5 * tr, hi = 0.5 * ti;
  const bool imag = (ti == 0.0);
  const int L = s.L();
  Ctx c = ctx();
  double t0;
  for (int k = 0; k < L && half != 2; ++k) {
    t0 = tic();
    site_update(s, k, hr, hi);
    toc(stats.t_site, t0);
    if (k < L - 1) {
      t0 = tic();
      shift_right(s, k, Kout_, Cb_);
      toc(stats.t_env, t0);
      t0 = tic();
      const int M = s.Mb[k + 1], Dw = H_.s[k].Dr;
      const cplx* Le = s.Lenv[k + 1];
      const cplx* Re = s.Renv[k];
      if (mixed() && M <= kFusedBondMaxM) {
        bond_exp(M, Dw, Le, Re, -hr, -hi);
      } else {
        if (mixed()) bond_tc_prepare(st_, tcb_, M, Dw, Le, Re);
        stats.bond_matvecs += krylov((long long)M * M, Cb_, Rb_, -hr, -hi,
                                     [&](const cplx* in, cplx* out, const int* sk) {
          if (mixed())
            bond_tc_apply(st_, tcb_, M, Dw, in, out);
          else
            bond_f64(c, M, Dw, Le, Re, in, out, sk);
        });
      }
      toc(stats.t_bond, t0);
      t0 = tic();
      absorb_left(Rb_, M, s.A[k + 1], (long long)s.D[k + 1] * s.Mb[k + 2]);
      if (imag) renormalize(s.A[k + 1], s.size(k + 1));
      toc(stats.t_absorb, t0);
    } else {
      CK(cudaMemcpyAsync(s.A[k], Kout_, sizeof(cplx) * (size_t)s.size(k),
                         cudaMemcpyDeviceToDevice, st_));
    }
  }
  for (int k = L - 1; k >= 0 && half != 1; --k) {
    t0 = tic();
    site_update(s, k, hr, hi);
    toc(stats.t_site, t0);
    if (k > 0) {
      t0 = tic();
      shift_left(s, k, Kout_, Cb_);
      toc(stats.t_env, t0);
      t0 = tic();
      const int M = s.Mb[k], Dw = H_.s[k].Dl;
      const cplx* Le = s.Lenv[k];
      const cplx* Re = s.Renv[k - 1];
      if (mixed() && M <= kFusedBondMaxM) {
        bond_exp(M, Dw, Le, Re, -hr, -hi);
      } else {
        if (mixed()) bond_tc_prepare(st_, tcb_, M, Dw, Le, Re);
        stats.bond_matvecs += krylov((long long)M * M, Cb_, Rb_, -hr, -hi,
                                     [&](const cplx* in, cplx* out, const int* sk) {
          if (mixed())
            bond_tc_apply(st_, tcb_, M, Dw, in, out);
          else
            bond_f64(c, M, Dw, Le, Re, in, out, sk);
        });
      }
      toc(stats.t_bond, t0);
      t0 = tic();
      absorb_right(s.A[k - 1], (long long)s.Mb[k - 1] * s.D[k - 1], Rb_, M);
      if (imag) renormalize(s.A[k - 1], s.size(k - 1));
      toc(stats.t_absorb, t0);
    } else {
      CK(cudaMemcpyAsync(s.A[k], Kout_, sizeof(cplx) * (size_t)s.size(k),
                         cudaMemcpyDeviceToDevice, st_));
    }
  }
}

// ------------------------------------------------------------------------------------
// observables and the application of j
// ------------------------------------------------------------------------------------
Cx Engine::overlap(const DevMps& bra, const DevMpo& W, const DevMps& ket) {
  const int L = bra.L();
  int cur = 0;
  set_ones(env_tmp_[0]);
  for (int k = 0; k < L; ++k) {
    env_left_any(W.s[k], bra.Mb[k], bra.Mb[k + 1], ket.Mb[k], ket.Mb[k + 1], bra.D[k], bra.d[k],
                 env_tmp_[cur], bra.A[k], ket.A[k], env_tmp_[cur ^ 1]);
    cur ^= 1;
  }
  cplx r;
  CK(cudaMemcpyAsync(&r, env_tmp_[cur], sizeof(cplx), cudaMemcpyDeviceToHost, st_));
  CK(cudaStreamSynchronize(st_));
  stats.d2h_bytes += sizeof(cplx);
  return Cx(r.x, r.y);
}

// phi ~ W|psi> at psi's bond dimensions by one-site variational fitting; psi has its center
// at site 0 and right-orthonormal sites 1..L-1; phi starts as a copy of psi.
void Engine::fit_apply(const DevMpo& W, const DevMps& psi, DevMps& phi, int sweeps) {
  copy_mps(psi, phi);
  const int L = psi.L();
  std::vector<cplx*> Lf(L, nullptr), Rf(L, nullptr);
  struct Guard {
    std::vector<cplx*>& a;
    std::vector<cplx*>& b;
    ~Guard() {
      for (auto* p : a)
        if (p) cudaFree(p);
      for (auto* p : b)
        if (p) cudaFree(p);
    }
  } guard{Lf, Rf};
  for (int k = 0; k < L; ++k) {
    CK(cudaMalloc(&Lf[k], sizeof(cplx) * (size_t)env_size(psi, k, W.s[k].Dl, true)));
    CK(cudaMalloc(&Rf[k], sizeof(cplx) * (size_t)env_size(psi, k, W.s[k].Dr, false)));
  }
  set_ones(Lf[0]);
  set_ones(Rf[L - 1]);
  Ctx c = ctx();
  for (int k = L - 1; k > 0; --k) {
    const int Ml = psi.Mb[k], Mr = psi.Mb[k + 1];
    env_right_any(W.s[k], Ml, Mr, Ml, Mr, psi.D[k], psi.d[k], Rf[k], phi.A[k], psi.A[k],
                  Rf[k - 1]);
  }
  const bool mx = mixed();
  auto heff_any = [&](int k, const cplx* in, cplx* out) {
    const int Ml = psi.Mb[k], Mr = psi.Mb[k + 1];
    if (mx) {
      heff_tc_prepare(st_, tcb_, Ml, Mr, W.s[k].Dl, W.s[k].Dr, Lf[k], Rf[k]);
      heff_tc_apply(st_, tcb_, W.s[k], Ml, Mr, psi.D[k], psi.d[k], in, out);
    } else {
      heff_f64(c, W.s[k], Ml, Mr, psi.D[k], psi.d[k], Lf[k], Rf[k], in, out, nullptr);
    }
  };
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int k = 0; k < L; ++k) {
      const int Ml = psi.Mb[k], Mr = psi.Mb[k + 1], D = psi.D[k], d = psi.d[k];
      heff_any(k, psi.A[k], Kout_);
      if (k < L - 1) {
        if (mx)
          left_partial_tc(st_, tcb_, W.s[k], Ml, Ml, D, d, Mr, Lf[k], psi.A[k], Y_);
        else
          left_partial_f64(c, W.s[k], Ml, Ml, D, d, Mr, Lf[k], psi.A[k], Y_, nullptr);
        gauge_qr_dev(Ml * D, Mr, qref(Kout_, Mr, 1, NOSPLIT, 0, 0), W.s[k].Dr * Mr,
                     qref(Y_, Mr, 1, Mr, (long long)Ml * D * Mr, 0), phi.A[k], Rb_);
        env_left_any(W.s[k], Ml, Mr, Ml, Mr, D, d, Lf[k], phi.A[k], psi.A[k], Lf[k + 1]);
      } else {
        CK(cudaMemcpyAsync(phi.A[k], Kout_, sizeof(cplx) * (size_t)psi.size(k),
                           cudaMemcpyDeviceToDevice, st_));
      }
    }
    for (int k = L - 1; k >= 0; --k) {
      const int Ml = psi.Mb[k], Mr = psi.Mb[k + 1], D = psi.D[k], d = psi.d[k];
      heff_any(k, psi.A[k], Kout_);
      if (k > 0) {
        if (mx)
          right_partial_tc(st_, tcb_, W.s[k], Ml, D, d, Mr, Mr, Rf[k], psi.A[k], Y_);
        else
          right_partial_f64(c, W.s[k], Ml, D, d, Mr, Mr, Rf[k], psi.A[k], Y_, nullptr);
        gauge_qr_dev(D * Mr, Ml, qref(Kout_, 1, (long long)D * Mr, NOSPLIT, 0, 1),
                     W.s[k].Dl * Ml, qref(Y_, 1, (long long)D * Mr, NOSPLIT, 0, 1), T1_, Rb_);
        CK(ztranspose(D * Mr, Ml, T1_, phi.A[k], 1, st_));
        env_right_any(W.s[k], Ml, Mr, Ml, Mr, D, d, Rf[k], phi.A[k], psi.A[k], Rf[k - 1]);
      } else {
        CK(cudaMemcpyAsync(phi.A[k], Kout_, sizeof(cplx) * (size_t)psi.size(k),
                           cudaMemcpyDeviceToDevice, st_));
      }
    }
  }
  check_status();
}

// ------------------------------------------------------------------------------------
// public flow
// ------------------------------------------------------------------------------------
void Engine::thermal_prepare(double beta, double dtau, int M) {
  if (!(beta > 0.0) || !(dtau > 0.0) || M < 2)
    throw Failure{TDMRG_ERR_ARG, "thermal_prepare: need beta > 0, dtau > 0, M >= 2"};
  const double nsf = beta / (2.0 * dtau);
  const long long nsteps = std::llround(nsf);
  if (std::fabs(nsteps * 2.0 * dtau - beta) > 1e-9 * std::max(1.0, beta) || nsteps < 1)
    throw Failure{TDMRG_ERR_ARG, "thermal_prepare: beta must be an even multiple of dtau"};
  prepared_ = false;
  rt_ready_ = false;
  CK(cudaMemsetAsync(status_, 0, 4 * sizeof(int), st_));
  alloc_mps(psi_b_, M);
  // |I> on the one-carrier sector
  const auto ent = identity_state_entries(P);
  int* d_ent = nullptr;
  size_t maxe = 0;
  for (auto& e : ent) maxe = std::max(maxe, e.size());
  CK(cudaMalloc(&d_ent, sizeof(int) * std::max<size_t>(maxe, 1)));
  for (int k = 0; k < psi_b_.L(); ++k) {
    CK(cudaMemcpy(d_ent, ent[k].data(), sizeof(int) * ent[k].size(), cudaMemcpyHostToDevice));
    stats.h2d_bytes += sizeof(int) * ent[k].size();
    CK(zfill_identity_mps(psi_b_.A[k], psi_b_.Mb[k], psi_b_.D[k], psi_b_.Mb[k + 1], d_ent,
                          (int)ent[k].size() / 3, st_));
    CK(cudaStreamSynchronize(st_));
  }
  cudaFree(d_ent);
  CK(cudaMemsetAsync(scal_ + 3, 0, sizeof(double), st_));
  right_canonicalize(psi_b_);
  check_status();
  double n2 = norm2_dev(psi_b_.A[0], psi_b_.size(0));
  logZ_ = std::log(n2);
  scale_dev(psi_b_.A[0], psi_b_.size(0), 1.0 / std::sqrt(n2));
  for (long long i = 0; i < nsteps; ++i) {
    tdvp_step(psi_b_, -dtau, 0.0);
    n2 = norm2_dev(psi_b_.A[0], psi_b_.size(0));
    if (!std::isfinite(n2) || n2 <= 0.0)
      throw Failure{TDMRG_ERR_NONFINITE, "non-finite norm in imaginary-time step"};
    logZ_ += std::log(n2);
    scale_dev(psi_b_.A[0], psi_b_.size(0), 1.0 / std::sqrt(n2));
  }
  // the renormalisations inside the sweeps
  CK(cudaMemcpyAsync(h_pinned_d_ + 2, scal_ + 3, sizeof(double), cudaMemcpyDeviceToHost, st_));
  CK(cudaStreamSynchronize(st_));
  logZ_ += h_pinned_d_[2];
  prepared_ = true;
}

void Engine::sync_twin_settings() {
  Engine& t = *twin_;
  if (t.precision_ != precision_) t.set_precision(precision_);
  t.ktol_ = ktol_;
  t.ktol_user_ = true;
  t.kmax_ = kmax_;
  t.fixed_k_ = fixed_k_;
  t.rank_tol_ = rank_tol_;
  t.rank_tol_user_ = true;
  t.prof_ = prof_;
  t.qr_.wait = qr_.wait;
  t.bs_.wait = bs_.wait;
}

// the twin's first state becomes a copy of src (an MPS of this engine, complete on src_stream)
// with its right environments built on the twin's stream
void Engine::adopt_state(const DevMps& src, cudaStream_t src_stream) {
  CK(cudaStreamSynchronize(src_stream));
  if (psi1_.A.size() != src.A.size() || psi1_.Mb != src.Mb) {
    clear_graphs();
    free_mps(psi1_);
    alloc_mps(psi1_, *std::max_element(src.Mb.begin(), src.Mb.end()));
    if (psi1_.Mb != src.Mb) throw Failure{TDMRG_ERR_STATE, "twin: bond dimensions differ"};
  }
  for (int k = 0; k < src.L(); ++k)
    CK(cudaMemcpyAsync(psi1_.A[k], src.A[k], sizeof(cplx) * (size_t)src.size(k),
                       cudaMemcpyDeviceToDevice, st_));
  build_right_envs(psi1_);
  CK(cudaStreamSynchronize(st_));
  prepared_ = true;
  rt_ready_ = true;
}

void Engine::realtime_init() {
  if (!prepared_) throw Failure{TDMRG_ERR_STATE, "realtime_init before thermal_prepare"};
  twin_on_ = false;
  copy_mps(psi_b_, psi1_);
  build_right_envs(psi1_);
  fit_apply(J_, psi_b_, psi2_, 2);
  build_right_envs(psi2_);
  CK(cudaStreamSynchronize(st_));
  if (concurrent_ && !graphs_) {
    if (!twin_) {
      twin_.reset(new Engine(P));
      twin_->concurrent_ = false;
      cudaStream_t ts = nullptr;
      CK(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
      twin_->own_stream_ = ts;
      twin_->st_ = ts;
    }
    sync_twin_settings();
    twin_->adopt_state(psi2_, st_);
    twin_on_ = true;
  }
  rt_ready_ = true;
}

void Engine::realtime_step(int nsteps, double dt) {
  if (!rt_ready_) throw Failure{TDMRG_ERR_STATE, "realtime_step before realtime_init"};
  if (nsteps < 0 || !(dt > 0.0)) throw Failure{TDMRG_ERR_ARG, "realtime_step: need dt > 0"};
  if (!twin_on_) {
    for (int i = 0; i < nsteps; ++i) {
      tdvp_step(psi1_, 0.0, -dt);
      tdvp_step(psi2_, 0.0, -dt);
    }
    return;
  }
  // two lanes: cooperative grids capped to half of the SMs so that both co-reside
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_));
  const int cap = std::max(8, sms / 2);
  const int cap0 = qr_gcap_, tcap0 = twin_->qr_gcap_;
  qr_gcap_ = cap;
  twin_->qr_gcap_ = cap;
  sync_twin_settings();
  std::exception_ptr err;
  Engine* tw = twin_.get();
  const int dev = dev_;
  try {
    for (int i = 0; i < nsteps; ++i) {
      std::thread lane([tw, dev, dt, &err] {
        try {
          CK(cudaSetDevice(dev));
          tw->tdvp_step(tw->psi1_, 0.0, -dt);
        } catch (...) {
          err = std::current_exception();
        }
      });
      try {
        tdvp_step(psi1_, 0.0, -dt);
      } catch (...) {
        lane.join();
        throw;
      }
      lane.join();
      if (err) std::rethrow_exception(err);
    }
  } catch (...) {
    qr_gcap_ = cap0;
    twin_->qr_gcap_ = tcap0;
    throw;
  }
  qr_gcap_ = cap0;
  twin_->qr_gcap_ = tcap0;
}

void Engine::realtime_observe(double* C, double* obs) {
  if (!rt_ready_) throw Failure{TDMRG_ERR_STATE, "realtime_observe before realtime_init"};
  // the twin's steps ended with a synchronisation of its stream: its state is complete
  const DevMps& second = twin_on_ ? twin_->psi1_ : psi2_;
  const double t0 = tic();
  const Cx c = overlap(psi1_, J_, second);
  toc(stats.t_observe, t0);
  if (!std::isfinite(c.real()) || !std::isfinite(c.imag()))
    throw Failure{TDMRG_ERR_NONFINITE, "non-finite C(t)"};
  C[0] = c.real();
  C[1] = c.imag();
  if (obs) {
    obs[0] = overlap(psi1_, I_, psi1_).real();
    obs[1] = overlap(second, I_, second).real();
    obs[2] = overlap(psi1_, H_, psi1_).real();
  }
}

Stats Engine::total_stats() const {
  Stats s = stats;
  if (twin_) {
    const Stats& t = twin_->stats;
    s.site_updates += t.site_updates;
    s.matvecs += t.matvecs;
    s.heff_flops += t.heff_flops;
    s.krylov_vectors += t.krylov_vectors;
    s.bond_matvecs += t.bond_matvecs;
    s.qrs += t.qrs;
    s.completions += t.completions;
    s.env_updates += t.env_updates;
    s.heff_ms += t.heff_ms;
    s.qr_ms += t.qr_ms;
    s.qr_flops += t.qr_flops;
    s.qr_bulk_ms += t.qr_bulk_ms;
    s.qr_bulk_flops += t.qr_bulk_flops;
    s.qr_bulk_n += t.qr_bulk_n;
    s.lz_ms += t.lz_ms;
    s.t_site += t.t_site;
    s.t_qr += t.t_qr;
    s.t_env += t.t_env;
    s.t_bond += t.t_bond;
    s.t_absorb += t.t_absorb;
    s.h2d_bytes += t.h2d_bytes;
    s.d2h_bytes += t.d2h_bytes;
    s.replayed_launches += t.replayed_launches;
  }
  return s;
}


// sigma_ij = <Psi_b| c+_j c_i |Psi_b> (Eq. 9; the ancilla and every phonon traced out), all N^2
// entries in one left-to-right pass of transfer contractions.  Psi_b is normalised with its
// center at site 0 and sites 1.. right-orthonormal, so the right transfer environment of every
// bond is the identity and an entry is the trace of a left environment.  Carried along the
// chain: the identity-transfer environment E and, for every molecule p already passed, the
// environments with c_p or c+_p inserted at its electronic site.  At the electronic site of
// molecule q each of those is closed with c+_q or c_q (one transfer and a trace), E gives the
// diagonal entry with n_q, and two new ones start from E.
void Engine::reduced_density(double* sigma) {
  if (!prepared_) throw Failure{TDMRG_ERR_STATE, "reduced_density before thermal_prepare"};
  const DevMps& s = psi_b_;
  const int L = s.L(), N = P.N;
  auto one_site = [](int which) {
    MpoSite m;
    m.Dl = m.Dr = 1;
    m.d = 2;
    std::vector<Cx> op(4, Cx(0, 0));
    if (which == 0) op[0 * 2 + 1] = Cx(1, 0);        // c  : |1> -> |0>
    else if (which == 1) op[1 * 2 + 0] = Cx(1, 0);   // c+ : |0> -> |1>
    else op[1 * 2 + 1] = Cx(1, 0);                   // n
    m.blocks.push_back({0, 0, op});
    return m;
  };
  DevMpo ops;
  upload_mpo({one_site(0), one_site(1), one_site(2)}, ops);
  long long maxe = 1;
  for (int k = 0; k <= L; ++k) maxe = std::max(maxe, (long long)s.Mb[k] * s.Mb[k]);
  const int nbuf = 2 * (2 * N + 1);
  std::vector<cplx*> buf(nbuf, nullptr);
  cplx* tr = nullptr;
  struct Guard {
    DevMpo& o;
    std::vector<cplx*>& b;
    cplx*& t;
    ~Guard() {
      free_mpo(o);
      for (cplx* p : b)
        if (p) cudaFree(p);
      if (t) cudaFree(t);
    }
  } guard{ops, buf, tr};
  for (auto& p : buf) CK(cudaMalloc(&p, sizeof(cplx) * (size_t)maxe));
  CK(cudaMalloc(&tr, sizeof(cplx) * (size_t)N * N));
  CK(cudaMemsetAsync(tr, 0, sizeof(cplx) * (size_t)N * N, st_));
  // slot 0: E; slots 1 + 2p, 2 + 2p: c_p and c+_p inserted; two banks (current, next)
  int bank = 0;
  auto slot = [&](int b, int i) { return buf[b * (2 * N + 1) + i]; };
  std::vector<char> open(2 * N + 1, 0);
  set_ones(slot(0, 0));
  open[0] = 1;
  const DevMpoSite& Cop = ops.s[0];
  const DevMpoSite& Cdag = ops.s[1];
  const DevMpoSite& Nop = ops.s[2];
  for (int k = 0; k < L; ++k) {
    const int Ml = s.Mb[k], Mr = s.Mb[k + 1], D = s.D[k], d = s.d[k];
    const bool elec = sites_[k].kind == SiteInfo::ELEC;
    const int q = sites_[k].mol;
    auto transfer = [&](const DevMpoSite& W, const cplx* in, cplx* out) {
      env_left_any(W, Ml, Mr, Ml, Mr, D, d, in, s.A[k], s.A[k], out);
    };
    // scratch for closings: slot 0 of the other bank is free until E is advanced below
    cplx* scratch = slot(bank ^ 1, 0);
    if (elec) {
      for (int p = 0; p < q; ++p) {
        // c_p ... c+_q: <c+_q c_p> = sigma_pq;  c+_p ... c_q: <c+_p c_q> = sigma_qp
        transfer(Cdag, slot(bank, 1 + 2 * p), scratch);
        CK(ztrace(scratch, Mr, tr + (size_t)p * N + q, st_));
        transfer(Cop, slot(bank, 2 + 2 * p), scratch);
        CK(ztrace(scratch, Mr, tr + (size_t)q * N + p, st_));
      }
      transfer(Nop, slot(bank, 0), scratch);
      CK(ztrace(scratch, Mr, tr + (size_t)q * N + q, st_));
    }
    // advance every open environment through site k (identity), start the two new ones
    for (int i = 0; i < 2 * N + 1; ++i)
      if (open[i]) transfer(I_.s[k], slot(bank, i), slot(bank ^ 1, i));
    if (elec) {
      transfer(Cop, slot(bank, 0), slot(bank ^ 1, 1 + 2 * q));
      transfer(Cdag, slot(bank, 0), slot(bank ^ 1, 2 + 2 * q));
      open[1 + 2 * q] = open[2 + 2 * q] = 1;
    }
    bank ^= 1;
  }
  std::vector<cplx> h((size_t)N * N);
  CK(cudaMemcpyAsync(h.data(), tr, sizeof(cplx) * h.size(), cudaMemcpyDeviceToHost, st_));
  CK(cudaStreamSynchronize(st_));
  stats.d2h_bytes += sizeof(cplx) * h.size();
  check_status();
  for (size_t e = 0; e < h.size(); ++e) {
    if (!std::isfinite(h[e].x) || !std::isfinite(h[e].y))
      throw Failure{TDMRG_ERR_NONFINITE, "non-finite reduced density matrix"};
    sigma[2 * e] = h[e].x;
    sigma[2 * e + 1] = h[e].y;
  }
}

}  // namespace tdmrg
