// Solver drivers: tensor Krylov-Schur (Algorithm 5 with U = V, X = Y) and
// HOOI (Section 6.1) for (1,2)-symmetric tensors.  The host code only
// sequences launches and reads a few scalars per outer iteration (the
// gradient test and the number of columns each block QR keeps); every
// arithmetic step runs in the library's kernels on the caller's stream.
#include <atomic>
#include <chrono>
#include <cmath>
#include <set>

#include "dense.cuh"

namespace bks {

namespace {

constexpr int kBasisCap = 128;   // k1, k3 <= 128 (inner solve limit)
constexpr int kBlockMax = 32;    // columns of one contraction result
constexpr int kInnerStartSweeps = 5;  // HOOI sweeps after the HOSVD start (Section 6.2)
constexpr int kFastHooiSweeps = 20;   // fast schedule: HOOI sweeps before Newton takes over

__global__ void k_f3w(const double* __restrict__ H1, int r1, int r3, double* __restrict__ F3wT) {
  // F3wT (w3 x r3, ld w3): row tri(a,b), column c = w_ab F[a,b,c], F[a,b,c] = H1[a + r1(b + r1 c)]
  const int w3 = r1 * (r1 + 1) / 2;
  for (int x = threadIdx.x; x < w3 * r3; x += blockDim.x) {
    const int t = x % w3, c = x / w3;
    int b = 0;
    while ((b + 1) * (b + 2) / 2 <= t) ++b;
    const int a = t - b * (b + 1) / 2;
    F3wT[x] = (a == b ? 1.0 : 2.0) * H1[a + r1 * (b + r1 * c)];
  }
}

__global__ void k_sumsq(const double* __restrict__ x, int n, double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], x[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_copy2d(const double* __restrict__ src, int64_t lds, int64_t rows, int cols,
                         double* __restrict__ dst, int64_t ldd) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % rows, c = t / rows;
    dst[r + ldd * c] = src[r + lds * c];
  }
}

// scale the off-diagonal triangle columns by sqrt(2): then T T^T equals the
// Gram of the full (a,b) unfolding
__global__ void k_tri_weight(double* __restrict__ T, int64_t n, int r1) {
  const int w3 = r1 * (r1 + 1) / 2;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n * w3;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(x / n);
    int b = 0;
    while ((b + 1) * (b + 2) / 2 <= t) ++b;
    const int a = t - b * (b + 1) / 2;
    if (a != b) T[x] *= 1.4142135623730951;
  }
}

// Refinement form of the core (mixed precision, FP64 phase): overwrite the
// blocks of C that carry first-order information at the current point
// (U, W) = (X[:, :r1], Z[:, :r3]) with FP64 values from the stage-1
// contractions:
//   C[x, b, c] = C[b, x, c] = (X^T A.(U,W)_{2,3})[x, b + r1 c]  (b < r1, c < r3)
//   C[a, b, c] = C[b, a, c] = (Z^T A.(U,U)_{1,2})[c, a + b(b+1)/2] (a <= b < r1, c >= r3)
// G1 = [X M1]^T M1 ((k1 + r1 r3) x r1 r3), G3 = [Z M3]^T M3 ((k3 + w3) x w3).
// Each entry is written by one thread only (x < r1 only when x <= b; the
// mode-3 block only where c >= r3), so the result is deterministic.
__global__ void k_core_patch(double* __restrict__ C, int k1, int k3, int r1, int r3,
                             const double* __restrict__ G1, const double* __restrict__ G3) {
  const int w1 = r1 * r3, w3 = r1 * (r1 + 1) / 2;
  const int n1 = k1 * w1, n3 = w3 * (k3 - r3);
  const int64_t kk = (int64_t)k1 * k1;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n1 + n3; o += gridDim.x * blockDim.x) {
    if (o < n1) {
      const int x = o % k1, j = o / k1, b = j % r1, c = j / r1;
      if (x < r1 && x > b) continue;
      const double v = G1[x + (int64_t)(k1 + w1) * j];
      C[x + (int64_t)k1 * b + kk * c] = v;
      C[b + (int64_t)k1 * x + kk * c] = v;
    } else {
      const int y = o - n1;
      const int c = r3 + y % (k3 - r3), t = y / (k3 - r3);
      int b = 0;
      while ((b + 1) * (b + 2) / 2 <= t) ++b;
      const int a = t - b * (b + 1) / 2;
      const double v = G3[c + (int64_t)(k3 + w3) * t];
      C[a + (int64_t)k1 * b + kk * c] = v;
      C[b + (int64_t)k1 * a + kk * c] = v;
    }
  }
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 32));
}

int copy2d(const double* src, int64_t lds, int64_t rows, int cols, double* dst, int64_t ldd,
           cudaStream_t s) {
  if (rows * cols == 0) return BKS_OK;
  k_copy2d<<<grid_for(rows * cols), 256, 0, s>>>(src, lds, rows, cols, dst, ldd); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

struct Block {
  int off = 0, width = 0;
};

struct PairSpec {
  int a, b;
  bool tri;
};

// Block pairs of one stage (Tables 1-3): U-pairs (left U block, right W
// block) then W-pairs (two U blocks; `tri` when both are the same block).
void stage_pairs(int variant, int stage, int nU, int nW, std::set<std::pair<int, int>>& doneU,
                 std::set<std::pair<int, int>>& doneW, std::vector<PairSpec>& us,
                 std::vector<PairSpec>& ws) {
  us.clear();
  ws.clear();
  if (stage == 1) {
    us.push_back({0, 0, false});
    ws.push_back({0, 0, true});
    return;
  }
  const int q = stage - 1;
  if (variant == BKS_VARIANT_BK) {
    if (q >= nU || q >= nW) return;
    for (int t = 0; t < q; ++t) {
      us.push_back({t, q, false});
      us.push_back({q, t, false});
    }
    for (int t = 0; t < q; ++t) ws.push_back({t, q, false});
  } else if (variant == BKS_VARIANT_MIN) {
    if (q >= nU || q >= nW) return;
    us.push_back({q, q, false});
    ws.push_back({q, q, true});
  } else {
    const int top = std::max(nU, nW);
    for (int sh = 0; sh < top; ++sh) {
      for (int t = 0; t < sh; ++t) {
        const int cand[2][2] = {{t, sh}, {sh, t}};
        for (auto& c : cand)
          if (c[0] < nU && c[1] < nW && !doneU.count({c[0], c[1]})) us.push_back({c[0], c[1], false});
      }
      if (sh < nU && sh < nW && !doneU.count({sh, sh})) us.push_back({sh, sh, false});
    }
    for (int sh = 0; sh < nU; ++sh)
      for (int t = 0; t <= sh; ++t)
        if (!doneW.count({t, sh})) ws.push_back({t, sh, t == sh});
  }
}

struct BksState {
  const bks_tensor* t = nullptr;
  cudaStream_t s = nullptr;
  int64_t m = 0, n = 0;
  int r1 = 0, r3 = 0;
  bks_params P{};
  DenseWork ws;
  DevBuf X, Z, H1, F3wT, C, Uh, Wh, negU, negW, inner_info, scal;
  // refinement form: FP64 stage-1 contractions kept for the core patch
  DevBuf M1raw, M3raw, G1, G3;
  bool keep_raw = false;
  int capX = 0, capZ = 0;
  int k1 = 0, k3 = 0;
  std::vector<Block> Ub, Wb;
  int inner_sweeps = 0;

  double* Xp() { return X.as<double>(); }
  double* Zp() { return Z.as<double>(); }

  int init(const bks_tensor* tt, const bks_params* prm, cudaStream_t st) {
    t = tt;
    s = st;
    P = *prm;
    m = t->m;
    n = t->n;
    r1 = P.r1;
    r3 = P.r3;
    capX = (int)std::min<int64_t>(m, kBasisCap);
    capZ = (int)std::min<int64_t>(n, kBasisCap);
    BKS_TRY(X.alloc(sizeof(double) * (size_t)m * (capX + kBlockMax), s));
    BKS_TRY(Z.alloc(sizeof(double) * (size_t)n * (capZ + kBlockMax), s));
    BKS_TRY(H1.alloc(sizeof(double) * (size_t)r1 * r1 * r3, s));
    BKS_TRY(F3wT.alloc(sizeof(double) * (size_t)r1 * (r1 + 1) / 2 * r3, s));
    BKS_TRY(C.alloc(sizeof(double) * (size_t)kBasisCap * kBasisCap * kBasisCap, s));
    BKS_TRY(Uh.alloc(sizeof(double) * kBasisCap * 8, s));
    BKS_TRY(Wh.alloc(sizeof(double) * kBasisCap * 8, s));
    BKS_TRY(negU.alloc(sizeof(double) * kBasisCap * 8, s));
    BKS_TRY(negW.alloc(sizeof(double) * kBasisCap * 8, s));
    BKS_TRY(inner_info.alloc(sizeof(double) * 8, s));
    BKS_TRY(scal.alloc(sizeof(double) * 8, s));
    if (P.precision == BKS_PREC_MIXED) {
      const int w1 = r1 * r3, w3 = r1 * (r1 + 1) / 2;
      BKS_TRY(M1raw.alloc(sizeof(double) * (size_t)m * w1, s));
      BKS_TRY(M3raw.alloc(sizeof(double) * (size_t)n * w3, s));
      BKS_TRY(G1.alloc(sizeof(double) * (size_t)(kBasisCap + kBlockMax) * w1, s));
      BKS_TRY(G3.alloc(sizeof(double) * (size_t)(kBasisCap + kBlockMax) * w3, s));
    }
    return BKS_OK;
  }

  int bar(int idx, const Block& b) const {
    if (P.variant == BKS_VARIANT_MAX || idx == 0) return b.width;
    return std::min(P.block_p, b.width);
  }

  // One U-block: mode-1 contraction of (Ub[a] bar, Wb[b] bar) into X after
  // the basis, then block QR against the basis.
  int add_u_block(int a, int b, bool fp32, bool stage1) {
    const int wl = bar(a, Ub[a]), wr = bar(b, Wb[b]);
    Block nb{k1, 0};
    if (wl == 0 || wr == 0) {
      Ub.push_back(nb);
      return BKS_OK;
    }
    if (wl > 8 || wr > 8 || wl * wr > kBlockMax)
      return fail(BKS_EUNSUPPORTED, "block contraction wider than 8 x 8 or 32 columns");
    double* dst = Xp() + (size_t)m * k1;
    BKS_TRY(contract_mode1_x(t, Xp() + (size_t)m * Ub[a].off, m, wl, Zp() + (size_t)n * Wb[b].off,
                             n, wr, dst, m, fp32, s));
    if (stage1 && keep_raw) BKS_TRY(copy2d(dst, m, m, wl * wr, M1raw.as<double>(), m, s));
    OrthOpts o;
    o.drop_tol = P.drop_tol;
    o.cap = capX - k1;
    o.two_level = true;
    o.fast_first = fp32;
    if (stage1) {
      o.grad_out = scal.as<double>() + 0;
      o.grad_mat = nullptr;  // H^T: the gradient weights are unfold_1(F) itself
      o.grad_cols = r1;
      o.h_out_early = H1.as<double>();
    }
    int bo = 0;
    BKS_TRY(orth_block(Xp(), m, k1, dst, m, wl * wr, m, o, nullptr, nullptr, &bo, ws, s));
    nb.width = bo;
    k1 += bo;
    Ub.push_back(nb);
    return BKS_OK;
  }

  int add_w_block(int a, int b, bool tri, bool fp32, bool stage1) {
    const int wl = bar(a, Ub[a]), wr = bar(b, Ub[b]);
    Block nb{k3, 0};
    if (wl == 0 || wr == 0) {
      Wb.push_back(nb);
      return BKS_OK;
    }
    const int w = tri ? wl * (wl + 1) / 2 : wl * wr;
    if (wl > 8 || wr > 8 || w > kBlockMax)
      return fail(BKS_EUNSUPPORTED, "block contraction wider than 8 x 8 or 32 columns");
    double* dst = Zp() + (size_t)n * k3;
    BKS_TRY(contract_mode3_x(t, Xp() + (size_t)m * Ub[a].off, m, wl,
                             tri ? nullptr : Xp() + (size_t)m * Ub[b].off, m, wr, dst, n, fp32, s));
    if (stage1 && keep_raw) BKS_TRY(copy2d(dst, n, n, w, M3raw.as<double>(), n, s));
    OrthOpts o;
    o.drop_tol = P.drop_tol;
    o.cap = capZ - k3;
    o.two_level = true;
    o.fast_first = fp32;
    if (stage1) {
      k_f3w<<<1, 256, 0, s>>>(H1.as<double>(), r1, r3, F3wT.as<double>()); ::bks::note_launch();
      BKS_CUDA_TRY(cudaGetLastError());
      o.grad_out = scal.as<double>() + 1;
      o.grad_mat = F3wT.as<double>();
      o.grad_cols = r3;
    }
    int bo = 0;
    BKS_TRY(orth_block(Zp(), n, k3, dst, n, w, n, o, nullptr, nullptr, &bo, ws, s));
    nb.width = bo;
    k3 += bo;
    Wb.push_back(nb);
    return BKS_OK;
  }

  // Stage 1 from (U0, W0) = (X[:, :r1], Z[:, :r3]); returns grad, ||F||.
  int stage1(bool fp32, double* grad, double* normF) {
    k1 = r1;
    k3 = r3;
    Ub.assign(1, Block{0, r1});
    Wb.assign(1, Block{0, r3});
    BKS_CUDA_TRY(cudaMemsetAsync(scal.p, 0, sizeof(double) * 4, s));
    BKS_TRY(add_u_block(0, 0, fp32, true));
    BKS_TRY(add_w_block(0, 0, true, fp32, true));
    k_sumsq<<<1, 256, 0, s>>>(H1.as<double>(), r1 * r1 * r3, scal.as<double>() + 2); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    double h[3];
    BKS_CUDA_TRY(cudaMemcpyAsync(h, scal.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    *grad = std::sqrt(std::max(0.0, 2.0 * h[0] + h[1]));
    *normF = std::sqrt(std::max(0.0, h[2]));
    return BKS_OK;
  }

  int expand_rest(bool fp32) {
    std::set<std::pair<int, int>> doneU{{0, 0}}, doneW{{0, 0}};
    std::vector<PairSpec> us, wsp;
    for (int st = 2; st <= P.stages; ++st) {
      stage_pairs(P.variant, st, (int)Ub.size(), (int)Wb.size(), doneU, doneW, us, wsp);
      for (auto& pr : us) {
        doneU.insert({pr.a, pr.b});
        BKS_TRY(add_u_block(pr.a, pr.b, fp32, false));
      }
      for (auto& pr : wsp) {
        doneW.insert({pr.a, pr.b});
        BKS_TRY(add_w_block(pr.a, pr.b, pr.tri, fp32, false));
      }
    }
    return BKS_OK;
  }

  double cur_tol = 0.0;  // outer tolerance of the current phase
  double last_nf = 1.0;  // ||F|| at the last stage-1 evaluation
  double last_grad_rel = 0.0;  // ||grad|| / ||F|| there

  // The core C = A.(X,X,Z); in the refinement form (keep_raw) computed in
  // FP32 and then patched with the FP64 first-order blocks.
  int core() {
    BKS_TRY(contract_core_x(t, Xp(), m, k1, Zp(), n, k3, C.as<double>(), fp32_core(), s));
    if (!keep_raw) return BKS_OK;
    const int w1 = r1 * r3, w3 = r1 * (r1 + 1) / 2;
    BKS_TRY(ts_gram(Xp(), m, k1, M1raw.as<double>(), m, w1, m, G1.as<double>(), ws, s));
    BKS_TRY(ts_gram(Zp(), n, k3, M3raw.as<double>(), n, w3, n, G3.as<double>(), ws, s));
    const int tot = k1 * w1 + w3 * (k3 - r3);
    k_core_patch<<<std::max(1, (tot + 255) / 256), 256, 0, s>>>(C.as<double>(), k1, k3, r1, r3,
                                                               G1.as<double>(), G3.as<double>());
    ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    return BKS_OK;
  }
  bool core_fp32 = false;
  bool fp32_core() const { return core_fp32 || keep_raw; }

  int last_k1 = 0, last_k3 = 0;  // basis sizes of the last expansion

  int inner_and_restart(bool fp32, cudaEvent_t* ev) {
    core_fp32 = fp32;
    last_k1 = k1;
    last_k3 = k3;
    BKS_TRY(core());
    BKS_CUDA_TRY(cudaEventRecord(ev[0], s));
    // inner tolerance (the inner test is ||grad_C|| / ||F_C||; with the
    // scale-free outer test the tolerance is carried over through ||F||).
    // BKS_INNER_PAPER (Section 6.2): the truncated HOSVD start gets 5 HOOI
    // sweeps, then Newton-Grassmann steps solve the inner problem to the
    // outer criterion.  BKS_INNER_FAST: no start sweeps, up to 20 HOOI
    // sweeps, then Newton-Grassmann, to an inexact tolerance a hundred
    // times below the current outer gradient and at least a tenth of the
    // outer tolerance.  inner_tol > 0 replaces either tolerance.
    const double otol = P.tol_scale_free ? cur_tol * last_nf : cur_tol;
    const bool fast = P.inner_schedule == BKS_INNER_FAST;
    const double itol = P.inner_tol > 0 ? P.inner_tol
                        : fast ? std::max(0.1 * otol, 0.01 * last_grad_rel) : otol;
    BKS_TRY(inner_solve(C.as<double>(), k1, k3, r1, r3, itol, P.max_inner,
                        fast ? 0 : kInnerStartSweeps, fast ? kFastHooiSweeps : 0,
                        Uh.as<double>(), Wh.as<double>(),
                        negU.as<double>(), negW.as<double>(), inner_info.as<double>(), s));
    BKS_CUDA_TRY(cudaEventRecord(ev[1], s));
    // U0 <- X Uh, W0 <- Z Wh (eq. (tks1)), in place in the first columns
    BKS_TRY(ts_combine(Xp(), m, k1, nullptr, m, 0, negU.as<double>(), nullptr, r1, Xp(), m, m,
                       ws, s));
    BKS_TRY(ts_combine(Zp(), n, k3, nullptr, n, 0, negW.as<double>(), nullptr, r3, Zp(), n, n,
                       ws, s));
    BKS_CUDA_TRY(cudaEventRecord(ev[2], s));
    double info[4];
    BKS_CUDA_TRY(cudaMemcpyAsync(info, inner_info.p, sizeof(info), cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    inner_sweeps += (int)info[2];
    return BKS_OK;
  }
};

int check_params(const bks_tensor* t, const bks_params* p) {
  if (!t || !p) return fail(BKS_EINVAL, "null tensor or params");
  BKS_TRY(require_symmetric(t));
  if (p->r1 < 1 || p->r3 < 1 || p->r1 > 8 || p->r3 > 8)
    return fail(BKS_EUNSUPPORTED, "ranks must be in 1..8");
  if (p->r1 > t->m || p->r3 > t->n) return fail(BKS_EINVAL, "rank larger than the dimension");
  if (p->r1 * p->r3 > kBlockMax) return fail(BKS_EUNSUPPORTED, "r1*r3 must be <= 32");
  if (p->stages < 1 || p->block_p < 1 || p->block_p > 8)
    return fail(BKS_EINVAL, "stages >= 1 and 1 <= block_p <= 8 required");
  if (p->variant < BKS_VARIANT_BK || p->variant > BKS_VARIANT_MAX)
    return fail(BKS_EINVAL, "unknown variant");
  if (p->precision != BKS_PREC_FP64 && p->precision != BKS_PREC_MIXED)
    return fail(BKS_EINVAL, "unknown precision");
  if (p->inner_schedule != BKS_INNER_PAPER && p->inner_schedule != BKS_INNER_FAST)
    return fail(BKS_EINVAL, "unknown inner schedule");
  return BKS_OK;
}

}  // namespace

}  // namespace bks

using namespace bks;

extern "C" void bks_params_default(bks_params* p) {
  if (!p) return;
  *p = bks_params{};
  p->r1 = 2;
  p->r3 = 2;
  p->stages = 2;
  p->block_p = 4;
  p->tol = 1e-10;
  p->max_outer = 500;
  p->max_inner = 1000;
  p->variant = BKS_VARIANT_BK;
  p->precision = BKS_PREC_FP64;
  p->refine_sweeps = 1;
  p->seed = 1;
  p->drop_tol = 1e-14;
  p->inner_tol = 0.0;
  p->mixed_tol = 1e-4;
  p->inner_schedule = BKS_INNER_PAPER;
}

extern "C" void hooi_params_default(hooi_params* p) {
  if (!p) return;
  *p = hooi_params{};
  p->r1 = 2;
  p->r3 = 2;
  p->tol = 1e-10;
  p->max_iter = 5000;
  p->grad_every = 10;
  p->precision = BKS_PREC_FP64;
  p->seed = 1;
  p->mixed_tol = 1e-4;
}

namespace bks {
int solve_impl(const bks_tensor* t, const bks_params* prm, const double* U0, const double* W0,
               double* U, double* W, double* F, bks_info* info, cudaStream_t stream,
               const std::atomic<int>* cancel);
}

extern "C" int bks_solve(const bks_tensor* t, const bks_params* prm, const double* U0,
                         const double* W0, double* U, double* W, double* F, bks_info* info,
                         void* stream) {
  return bks::solve_impl(t, prm, U0, W0, U, W, F, info, (cudaStream_t)stream, nullptr);
}

int bks::solve_impl(const bks_tensor* t, const bks_params* prm, const double* U0,
                    const double* W0, double* U, double* W, double* F, bks_info* info,
                    cudaStream_t stream, const std::atomic<int>* cancel) {
  BKS_TRY(check_params(t, prm));
  if (!U || !W || !F) return fail(BKS_EINVAL, "null output");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  BksState S;
  BKS_TRY(S.init(t, prm, s));
  const int64_t m = S.m, n = S.n;
  const int r1 = S.r1, r3 = S.r3;
  if (U0) BKS_TRY(copy2d(U0, m, m, r1, S.Xp(), m, s));
  else BKS_TRY(random_orthonormal(prm->seed, 1, m, r1, S.Xp(), S.ws, s));
  if (W0) BKS_TRY(copy2d(W0, n, n, r3, S.Zp(), n, s));
  else BKS_TRY(random_orthonormal(prm->seed, 3, n, r3, S.Zp(), S.ws, s));

  const bool mixed = prm->precision == BKS_PREC_MIXED;
  const double mtol = prm->mixed_tol > 0 ? prm->mixed_tol : 1e-4;
  bool fp32 = mixed;
  int it = 0, fp32_iters = 0, refine_left = std::max(0, prm->refine_sweeps);
  double grad = 0, nf = 0;
  bool converged = false;
  int status = BKS_OK;
  int hist_len = 0;
  double best_grad = INFINITY;
  int stall = 0;
  // phase timing with events on the stream (read after each iteration's
  // own synchronisation, so it adds no extra wait)
  cudaEvent_t ev[6];
  for (auto& e : ev) BKS_CUDA_TRY(cudaEventCreate(&e));
  double phase[5] = {0, 0, 0, 0, 0};
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() { for (int q = 0; q < 6; ++q) cudaEventDestroy(e[q]); }
  } evguard{ev};
  for (;; ++it) {
    if (cancel && cancel->load(std::memory_order_relaxed)) {
      status = fail(BKS_ECANCELED, "solve cancelled");
      break;
    }
    BKS_CUDA_TRY(cudaEventRecord(ev[0], s));
    // mixed precision after the FP32 phase: the refinement form (FP64
    // stage 1, FP32 expansion and core, FP64 first-order core blocks)
    S.keep_raw = mixed && !fp32;
    BKS_TRY(S.stage1(fp32, &grad, &nf));
    BKS_CUDA_TRY(cudaEventRecord(ev[1], s));
    // the stopping test: ||grad|| / ||F|| (Section 6.2) or the scale-free
    // ||grad|| / ||F||^2
    const double rel = nf > 0 ? (prm->tol_scale_free ? grad / (nf * nf) : grad / nf) : INFINITY;
    if (info && info->history && hist_len < info->history_cap) {
      info->history[2 * hist_len] = rel;
      info->history[2 * hist_len + 1] = nf;
      ++hist_len;
    }
    if (!std::isfinite(grad) || !std::isfinite(nf)) {
      status = fail(BKS_ENUMERIC, "NaN or Inf in the gradient or ||F||");
      break;
    }
    if (fp32) {
      // FP32-contraction phase: until the scale-free gradient
      // ||grad|| / ||F||^2 is below mixed_tol, or it stops halving for two
      // outer iterations (the FP32 noise floor); then FP64 refinement
      const double sf = nf > 0 ? grad / (nf * nf) : INFINITY;
      if (sf < best_grad * 0.5) { best_grad = sf; stall = 0; } else ++stall;
      if (sf <= mtol || stall >= 2 || rel <= prm->tol) {
        fp32 = false;
        continue;  // re-evaluate at the same point with FP64 contractions
      }
      ++fp32_iters;
    } else {
      if (rel <= prm->tol) { converged = true; break; }
      if (mixed && refine_left-- <= 0) break;
    }
    if (it >= prm->max_outer) break;
    S.cur_tol = fp32 ? (prm->tol_scale_free ? mtol : mtol * nf) : prm->tol;
    S.last_nf = nf;
    S.last_grad_rel = nf > 0 ? grad / nf : 0.0;
    BKS_TRY(S.expand_rest(fp32 || S.keep_raw));
    BKS_CUDA_TRY(cudaEventRecord(ev[2], s));
    BKS_TRY(S.inner_and_restart(fp32, ev + 3));
    {
      float ms;
      for (int q = 0; q < 5; ++q) {
        BKS_CUDA_TRY(cudaEventElapsedTime(&ms, ev[q], ev[q + 1]));
        phase[q] += ms;
      }
    }
  }
  // outputs: the point whose gradient was evaluated last
  BKS_TRY(copy2d(S.Xp(), m, m, r1, U, m, s));
  BKS_TRY(copy2d(S.Zp(), n, n, r3, W, n, s));
  BKS_TRY(copy2d(S.H1.as<double>(), r1, r1, r1 * r3, F, r1, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = it;
    info->converged = converged ? 1 : 0;
    info->grad_rel = nf > 0 ? (prm->tol_scale_free ? grad / (nf * nf) : grad / nf) : INFINITY;
    info->normF = nf;
    info->k1 = S.last_k1 ? S.last_k1 : S.k1;
    info->k3 = S.last_k3 ? S.last_k3 : S.k3;
    info->inner_sweeps = S.inner_sweeps;
    info->fp32_iters = fp32_iters;
    info->history_len = hist_len;
    for (int q = 0; q < 5; ++q) info->phase_ms[q] = phase[q];
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status != BKS_OK) return status;
  if (!converged) return fail(BKS_ENOTCONV, "not converged within the iteration limits");
  return BKS_OK;
}

// ---- HOOI -----------------------------------------------------------------
namespace bks {
namespace {

// ||T M - Q (Q^T T M)||_F^2 given Mq = Q^T T M precomputed: here we use the
// direct form ||T M - Q N||^2 with N = F F^T from the Gram of [Q T]^T T.
__global__ void k_hooi_small(const double* __restrict__ G, int K, int w, double* __restrict__ FT,
                             double* __restrict__ FF, double* __restrict__ nf2) {
  // G is the (K+w) x w Gram [Q T]^T T; F = G[0:K, :] (K x w)
  const int gw = K + w;
  for (int x = threadIdx.x; x < w * K; x += blockDim.x) {
    const int j = x % w, a = x / w;
    FT[j + w * a] = G[a + gw * j];  // F^T (w x K)
  }
  for (int x = threadIdx.x; x < K * K; x += blockDim.x) {
    const int a = x % K, b = x / K;
    double s = 0.0;
    for (int j = 0; j < w; ++j) s += G[a + gw * j] * G[b + gw * j];
    FF[x] = s;
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int a = 0; a < K; ++a)
      for (int j = 0; j < w; ++j) s += G[a + gw * j] * G[a + gw * j];
    *nf2 = s;
  }
}

__global__ void k_transpose(const double* __restrict__ A, int rows, int cols, double* __restrict__ B) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < rows * cols; x += gridDim.x * blockDim.x) {
    const int i = x % rows, j = x / rows;
    B[j + cols * i] = A[x];
  }
}
__global__ void k_trace_out(const double* __restrict__ G, int K, int g, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int j = 0; j < g; ++j) s += G[K + j + (int64_t)(K + g) * j];
    *out = s;
  }
}

}  // namespace

// tall-skinny helpers with Gram output (dense.cu internals re-exposed here
// through ts_combine + a Gram pass built from orth_block's machinery)
int ts_combine_gram(const double* Q, int64_t ldq, int K, const double* B, int64_t ldb, int b,
                    const double* Mq, const double* Mb, int bo, double* Out, int64_t ldo,
                    int64_t m, double* G, DenseWork& ws, cudaStream_t s);

}  // namespace bks


extern "C" int hooi_solve(const bks_tensor* t, const hooi_params* prm, const double* U0,
                          const double* W0, double* U, double* W, double* F, bks_info* info,
                          void* stream) {
  if (!t || !prm) return fail(BKS_EINVAL, "null tensor or params");
  BKS_TRY(require_symmetric(t));
  if (!U || !W || !F) return fail(BKS_EINVAL, "null output");
  const int r1 = prm->r1, r3 = prm->r3;
  if (r1 < 1 || r3 < 1 || r1 > 8 || r3 > 8 || r1 * r3 > kBlockMax)
    return fail(BKS_EUNSUPPORTED, "ranks must be in 1..8 with r1*r3 <= 32");
  if (r1 > t->m || r3 > t->n) return fail(BKS_EINVAL, "rank larger than the dimension");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t m = t->m, n = t->n;
  if (prm->precision != BKS_PREC_FP64 && prm->precision != BKS_PREC_MIXED)
    return fail(BKS_EINVAL, "unknown precision");
  // mixed precision: FP32 contractions until the FP32-evaluated gradient is
  // below mixed_tol (scale-free) or stops halving, then FP64 to the end
  bool fp32 = prm->precision == BKS_PREC_MIXED;
  const double mtol = prm->mixed_tol > 0 ? prm->mixed_tol : 1e-4;
  double best_sf = INFINITY;
  int stall = 0, fp32_iters = 0;
  bool force_check = false;
  const int w1 = r1 * r3, w3 = r1 * (r1 + 1) / 2;
  DenseWork ws;
  DevBuf Ub, Wb, T1, T3, T3c, G, FT, FF, FT3, FF3, sc, gout, gout3;
  BKS_TRY(Ub.alloc(sizeof(double) * m * r1, s));
  BKS_TRY(Wb.alloc(sizeof(double) * n * r3, s));
  BKS_TRY(T1.alloc(sizeof(double) * m * w1, s));
  BKS_TRY(T3.alloc(sizeof(double) * n * w3, s));
  BKS_TRY(T3c.alloc(sizeof(double) * n * w3, s));
  BKS_TRY(G.alloc(sizeof(double) * (kBlockMax + 8) * kBlockMax, s));
  BKS_TRY(FT.alloc(sizeof(double) * kBlockMax * 8, s));
  BKS_TRY(FF.alloc(sizeof(double) * 64, s));
  BKS_TRY(FT3.alloc(sizeof(double) * kBlockMax * 8, s));
  BKS_TRY(FF3.alloc(sizeof(double) * 64, s));
  BKS_TRY(sc.alloc(sizeof(double) * 8, s));
  BKS_TRY(gout.alloc(sizeof(double) * (size_t)m * r1, s));
  BKS_TRY(gout3.alloc(sizeof(double) * (size_t)n * r3, s));
  double* Up = Ub.as<double>();
  double* Wp = Wb.as<double>();
  if (U0) BKS_TRY(copy2d(U0, m, m, r1, Up, m, s));
  else BKS_TRY(random_orthonormal(prm->seed, 1, m, r1, Up, ws, s));
  if (W0) BKS_TRY(copy2d(W0, n, n, r3, Wp, n, s));
  else BKS_TRY(random_orthonormal(prm->seed, 3, n, r3, Wp, ws, s));
  auto make_t3 = [&]() -> int {
    BKS_TRY(contract_mode3_x(t, Up, m, r1, nullptr, m, r1, T3.as<double>(), n, fp32, s));
    k_tri_weight<<<grid_for(n * w3), 256, 0, s>>>(T3.as<double>(), n, r1); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    return BKS_OK;
  };
  BKS_TRY(make_t3());
  const int every = std::max(1, prm->grad_every);
  int it = 0;
  double grad = INFINITY, nf = 0;
  bool converged = false;
  int hist_len = 0;
  for (;; ++it) {
    BKS_TRY(contract_mode1_x(t, Up, m, r1, Wp, n, r3, T1.as<double>(), m, fp32, s));
    if (fp32) ++fp32_iters;
    if (it % every == 0 || it >= prm->max_iter || force_check) {
      force_check = false;
      // mode 1: F1 = U^T T1, gradient T1 F1^T - U (F1 F1^T)
      BKS_TRY(ts_gram(Up, m, r1, T1.as<double>(), m, w1, m, G.as<double>(), ws, s));
      k_hooi_small<<<1, 128, 0, s>>>(G.as<double>(), r1, w1, FT.as<double>(), FF.as<double>(),
                                     sc.as<double>() + 2); ::bks::note_launch();
      BKS_TRY(ts_combine_gram(Up, m, r1, T1.as<double>(), m, w1, FF.as<double>(), FT.as<double>(),
                              r1, gout.as<double>(), m, m, G.as<double>(), ws, s));
      k_trace_out<<<1, 32, 0, s>>>(G.as<double>(), r1, r1, sc.as<double>() + 0); ::bks::note_launch();
      // mode 3 with the weighted triangle T3w: F3w = W^T T3w
      BKS_TRY(ts_gram(Wp, n, r3, T3.as<double>(), n, w3, n, G.as<double>(), ws, s));
      k_hooi_small<<<1, 128, 0, s>>>(G.as<double>(), r3, w3, FT3.as<double>(), FF3.as<double>(),
                                     sc.as<double>() + 3); ::bks::note_launch();
      BKS_TRY(ts_combine_gram(Wp, n, r3, T3.as<double>(), n, w3, FF3.as<double>(),
                              FT3.as<double>(), r3, gout3.as<double>(), n, n, G.as<double>(), ws,
                              s));
      k_trace_out<<<1, 32, 0, s>>>(G.as<double>(), r3, r3, sc.as<double>() + 1); ::bks::note_launch();
      BKS_CUDA_TRY(cudaGetLastError());
      double h[4];
      BKS_CUDA_TRY(cudaMemcpyAsync(h, sc.p, sizeof(h), cudaMemcpyDeviceToHost, s));
      BKS_CUDA_TRY(cudaStreamSynchronize(s));
      grad = std::sqrt(std::max(0.0, 2.0 * h[0] + h[1]));
      nf = std::sqrt(std::max(0.0, h[2]));
      const double rel = nf > 0 ? grad / nf : INFINITY;
      if (info && info->history && hist_len < info->history_cap) {
        info->history[2 * hist_len] = rel;
        info->history[2 * hist_len + 1] = nf;
        ++hist_len;
      }
      if (!std::isfinite(grad)) return fail(BKS_ENUMERIC, "NaN or Inf in the gradient");
      if (fp32) {
        const double sf = nf > 0 ? grad / (nf * nf) : INFINITY;
        if (sf < 0.5 * best_sf) { best_sf = sf; stall = 0; } else ++stall;
        if (sf <= mtol || stall >= 2 || rel <= prm->tol) {
          // FP64 from here on: the contractions at the current point again,
          // and the gradient test on them at the next iteration
          fp32 = false;
          force_check = true;
          BKS_TRY(make_t3());
          --fp32_iters;
          continue;
        }
      } else {
        if (rel <= prm->tol) { converged = true; break; }
      }
      if (it >= prm->max_iter) break;
    }
    // U <- r1 leading left singular vectors of T1; W from the new U
    BKS_TRY(top_left_singular(T1.as<double>(), m, m, w1, r1, Up, m, ws, s));
    BKS_TRY(make_t3());
    BKS_TRY(copy2d(T3.as<double>(), n, n, w3, T3c.as<double>(), n, s));
    BKS_TRY(top_left_singular(T3c.as<double>(), n, n, w3, r3, Wp, n, ws, s));
  }
  // outputs: F = U^T T1 from the last gradient evaluation (FT holds F^T,
  // w1 x r1), written as unfold_1(F) = r1 x w1
  k_transpose<<<grid_for((int64_t)w1 * r1), 256, 0, s>>>(FT.as<double>(), w1, r1, F); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  BKS_TRY(copy2d(Up, m, m, r1, U, m, s));
  BKS_TRY(copy2d(Wp, n, n, r3, W, n, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = it;
    info->converged = converged ? 1 : 0;
    info->grad_rel = nf > 0 ? grad / nf : INFINITY;
    info->normF = nf;
    info->k1 = r1;
    info->k3 = r3;
    info->inner_sweeps = 0;
    info->fp32_iters = fp32_iters;
    for (int q = 0; q < 5; ++q) info->phase_ms[q] = 0.0;
    info->history_len = hist_len;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!converged) return fail(BKS_ENOTCONV, "HOOI not converged within max_iter");
  return BKS_OK;
}
