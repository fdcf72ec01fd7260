// Tensor Krylov-Schur for a general l x m x n tensor (Algorithm 5 as stated
// in Section 5): three bases X, Y, Z grown by the block-Krylov step of
// Algorithm 3 in each mode, the G-gradient from the stage-1 blocks by
// Proposition 2 (three terms), the core C = A.(X,Y,Z) (eq. (tkd)), the
// inner best rank-(r1,r2,r3) solve of C and the restart U = X Uh,
// V = Y Vh, W = Z Wh (eq. (tks1)).  FP64 throughout.  The host sequences
// launches and reads the gradient and the kept column counts once per
// outer iteration.
//
// Block schedules (the paper tabulates them for the (1,2)-symmetric case
// only; this library's general form): stage 1 makes U1 from (V0, W0), V1
// from (U0, W0), W1 from (U0, V0).  BK, stage t >= 2 with q = t - 1: each
// mode takes the pairs (0, q), (q, 0), ..., (q-1, q), (q, q-1) of the other
// two modes' blocks, the first p columns of each block except block 0;
// min-BK: the pair (t-1, t-1); max-BK: every unused pair of whole blocks,
// by shells.  Within a stage the mode-1 blocks come first, then mode 2,
// then mode 3, from the blocks that existed when the stage began.
#include <chrono>
#include <cmath>
#include <set>
#include <vector>

#include "dense.cuh"

namespace bks {

namespace {

constexpr int kGenCap = 128;        // k1, k2, k3 <= 128 (inner solve limit)
constexpr int kGenBlockMax = 32;    // columns of one contraction result
constexpr int kGenStartSweeps = 5;  // HOOI sweeps after the HOSVD start (Section 6.2)

__global__ void k_gsumsq(const double* __restrict__ x, int n, double* __restrict__ out) {
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

__global__ void k_gcopy2d(const double* __restrict__ src, int64_t lds, int64_t rows, int cols,
                          double* __restrict__ dst, int64_t ldd) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % rows, c = t / rows;
    dst[r + ldd * c] = src[r + lds * c];
  }
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 32));
}

int gcopy2d(const double* src, int64_t lds, int64_t rows, int cols, double* dst, int64_t ldd,
            cudaStream_t s) {
  if (rows * cols == 0) return BKS_OK;
  k_gcopy2d<<<grid_for(rows * cols), 256, 0, s>>>(src, lds, rows, cols, dst, ldd); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

struct GBlock {
  int off = 0, width = 0;
};
using PairSet = std::set<std::pair<int, int>>;

// Pairs (left, right) of one stage for mode md (0, 1, 2): mode 1 pairs
// (V, W) blocks, mode 2 (U, W), mode 3 (U, V); na, nb blocks of the two.
void gen_pairs(int variant, int stage, int na, int nb, const PairSet& done,
               std::vector<std::pair<int, int>>& out) {
  out.clear();
  if (stage == 1) {
    out.push_back({0, 0});
    return;
  }
  const int q = stage - 1;
  if (variant == BKS_VARIANT_BK) {
    if (q >= na || q >= nb) return;
    for (int t = 0; t < q; ++t) {
      out.push_back({t, q});
      out.push_back({q, t});
    }
  } else if (variant == BKS_VARIANT_MIN) {
    if (q < na && q < nb) out.push_back({q, q});
  } else {
    for (int sh = 0; sh < std::max(na, nb); ++sh) {
      for (int t = 0; t < sh; ++t) {
        const std::pair<int, int> cand[2] = {{t, sh}, {sh, t}};
        for (auto& c : cand)
          if (c.first < na && c.second < nb && !done.count(c)) out.push_back(c);
      }
      if (sh < na && sh < nb && !done.count({sh, sh})) out.push_back({sh, sh});
    }
  }
}

struct GenState {
  const bks_tensor* t = nullptr;
  cudaStream_t s = nullptr;
  int64_t dim[3] = {0, 0, 0};
  int r[3] = {0, 0, 0};
  bks_gen_params P{};
  DenseWork ws;
  DevBuf B[3], neg[3], C, H1, inner_info, scal;
  int cap[3] = {0, 0, 0}, k[3] = {0, 0, 0};
  std::vector<GBlock> blocks[3];
  int inner_sweeps = 0;
  int last_k[3] = {0, 0, 0};

  double* Bp(int md) { return B[md].as<double>(); }

  int init(const bks_tensor* tt, const bks_gen_params* prm, cudaStream_t st) {
    t = tt;
    s = st;
    P = *prm;
    dim[0] = t->l; dim[1] = t->m; dim[2] = t->n;
    r[0] = P.r1; r[1] = P.r2; r[2] = P.r3;
    for (int md = 0; md < 3; ++md) {
      cap[md] = (int)std::min<int64_t>(dim[md], kGenCap);
      BKS_TRY(B[md].alloc(sizeof(double) * (size_t)dim[md] * (cap[md] + kGenBlockMax), s));
      BKS_TRY(neg[md].alloc(sizeof(double) * kGenCap * 8, s));
    }
    BKS_TRY(C.alloc(sizeof(double) * (size_t)kGenCap * kGenCap * kGenCap, s));
    BKS_TRY(H1.alloc(sizeof(double) * (size_t)r[0] * r[1] * r[2], s));
    BKS_TRY(inner_info.alloc(sizeof(double) * 8, s));
    BKS_TRY(scal.alloc(sizeof(double) * 8, s));
    return BKS_OK;
  }

  int bar(int idx, const GBlock& b) const {
    if (P.variant == BKS_VARIANT_MAX || idx == 0) return b.width;
    return std::min(P.block_p, b.width);
  }

  // One block of mode md from blocks a, b of the other two modes: the
  // contraction into the columns after the basis, then block QR against it
  // (with the stage-1 gradient term ||P H^T||^2 to scal[md]).
  int add_block(int md, int a, int b, bool stage1) {
    static const int oth[3][2] = {{1, 2}, {0, 2}, {0, 1}};
    const int oa = oth[md][0], ob = oth[md][1];
    const int wl = bar(a, blocks[oa][a]), wr = bar(b, blocks[ob][b]);
    GBlock nb{k[md], 0};
    if (wl == 0 || wr == 0) {
      blocks[md].push_back(nb);
      return BKS_OK;
    }
    if (wl > 8 || wr > 8 || wl * wr > kGenBlockMax)
      return fail(BKS_EUNSUPPORTED, "block contraction wider than 8 x 8 or 32 columns");
    const int64_t d = dim[md];
    double* dst = Bp(md) + (size_t)d * k[md];
    BKS_TRY(gen_contract_x(t, md + 1, Bp(oa) + (size_t)dim[oa] * blocks[oa][a].off, dim[oa], wl,
                           Bp(ob) + (size_t)dim[ob] * blocks[ob][b].off, dim[ob], wr, dst, d, s));
    OrthOpts o;
    o.drop_tol = P.drop_tol;
    o.cap = cap[md] - k[md];
    o.two_level = true;
    if (stage1) {
      o.grad_out = scal.as<double>() + md;
      o.grad_mat = nullptr;  // M = H^T: H = Q^T B is unfold_md(F)
      o.grad_cols = r[md];
      if (md == 0) o.h_out_early = H1.as<double>();
    }
    int bo = 0;
    BKS_TRY(orth_block(Bp(md), d, k[md], dst, d, wl * wr, d, o, nullptr, nullptr, &bo, ws, s));
    nb.width = bo;
    k[md] += bo;
    blocks[md].push_back(nb);
    return BKS_OK;
  }

  int stage1(double* grad, double* normF) {
    for (int md = 0; md < 3; ++md) {
      k[md] = r[md];
      blocks[md].assign(1, GBlock{0, r[md]});
    }
    BKS_CUDA_TRY(cudaMemsetAsync(scal.p, 0, sizeof(double) * 4, s));
    for (int md = 0; md < 3; ++md) BKS_TRY(add_block(md, 0, 0, true));
    k_gsumsq<<<1, 256, 0, s>>>(H1.as<double>(), r[0] * r[1] * r[2], scal.as<double>() + 3); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    double h[4];
    BKS_CUDA_TRY(cudaMemcpyAsync(h, scal.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    *grad = std::sqrt(std::max(0.0, h[0] + h[1] + h[2]));
    *normF = std::sqrt(std::max(0.0, h[3]));
    return BKS_OK;
  }

  int expand_rest() {
    PairSet done[3];
    for (auto& d : done) d.insert({0, 0});
    static const int oth[3][2] = {{1, 2}, {0, 2}, {0, 1}};
    std::vector<std::pair<int, int>> pairs[3];
    for (int st = 2; st <= P.stages; ++st) {
      // every pair of the stage from the blocks at its start
      int nblk[3];
      for (int md = 0; md < 3; ++md) nblk[md] = (int)blocks[md].size();
      for (int md = 0; md < 3; ++md)
        gen_pairs(P.variant, st, nblk[oth[md][0]], nblk[oth[md][1]], done[md], pairs[md]);
      for (int md = 0; md < 3; ++md)
        for (auto& pr : pairs[md]) {
          done[md].insert(pr);
          BKS_TRY(add_block(md, pr.first, pr.second, false));
        }
    }
    return BKS_OK;
  }

  int inner_and_restart(double itol, int start_sweeps) {
    for (int md = 0; md < 3; ++md) last_k[md] = k[md];
    BKS_TRY(gen_core_x(t, Bp(0), dim[0], k[0], Bp(1), dim[1], k[1], Bp(2), dim[2], k[2],
                       C.as<double>(), s));
    BKS_TRY(gen_inner_solve(C.as<double>(), k[0], k[1], k[2], r[0], r[1], r[2], itol,
                            P.max_inner, start_sweeps, neg[0].as<double>(),
                            neg[1].as<double>(), neg[2].as<double>(), inner_info.as<double>(), s));
    // U0 <- X Uh, V0 <- Y Vh, W0 <- Z Wh (eq. (tks1)), in place
    for (int md = 0; md < 3; ++md)
      BKS_TRY(ts_combine(Bp(md), dim[md], k[md], nullptr, dim[md], 0, neg[md].as<double>(), nullptr,
                         r[md], Bp(md), dim[md], dim[md], ws, s));
    double info[4];
    BKS_CUDA_TRY(cudaMemcpyAsync(info, inner_info.p, sizeof(info), cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    inner_sweeps += (int)info[2];
    return BKS_OK;
  }
};

int check_gen_params(const bks_tensor* t, const bks_gen_params* p) {
  if (!t || !p) return fail(BKS_EINVAL, "null tensor or params");
  BKS_TRY(require_general(t));
  const int r[3] = {p->r1, p->r2, p->r3};
  const int64_t d[3] = {t->l, t->m, t->n};
  for (int md = 0; md < 3; ++md) {
    if (r[md] < 1 || r[md] > 8) return fail(BKS_EUNSUPPORTED, "ranks must be in 1..8");
    if (r[md] > d[md]) return fail(BKS_EINVAL, "rank larger than the dimension");
  }
  if (p->r1 * p->r2 > kGenBlockMax || p->r1 * p->r3 > kGenBlockMax || p->r2 * p->r3 > kGenBlockMax)
    return fail(BKS_EUNSUPPORTED, "products of two ranks must be <= 32");
  if (p->stages < 1 || p->block_p < 1 || p->block_p > 8)
    return fail(BKS_EINVAL, "stages >= 1 and 1 <= block_p <= 8 required");
  if (p->variant < BKS_VARIANT_BK || p->variant > BKS_VARIANT_MAX)
    return fail(BKS_EINVAL, "unknown variant");
  if (p->inner_schedule != BKS_INNER_PAPER && p->inner_schedule != BKS_INNER_FAST)
    return fail(BKS_EINVAL, "unknown inner schedule");
  return BKS_OK;
}

// From G = [Q T]^T T ((K + w) x w, F = Q^T T its first K rows): FT = F^T
// (w x K), FF = F F^T (K x K) and nf2 = ||F||^2.
__global__ void k_gh_small(const double* __restrict__ G, int K, int w, double* __restrict__ FT,
                           double* __restrict__ FF, double* __restrict__ nf2) {
  const int gw = K + w;
  for (int x = threadIdx.x; x < w * K; x += blockDim.x) {
    const int j = x % w, a = x / w;
    FT[j + w * a] = G[a + gw * j];
  }
  for (int x = threadIdx.x; x < K * K; x += blockDim.x) {
    const int a = x % K, b = x / K;
    double s = 0.0;
    for (int j = 0; j < w; ++j) s = fma(G[a + gw * j], G[b + gw * j], s);
    FF[x] = s;
  }
  if (threadIdx.x == 0 && nf2) {
    double s = 0.0;
    for (int a = 0; a < K; ++a)
      for (int j = 0; j < w; ++j) s = fma(G[a + gw * j], G[a + gw * j], s);
    *nf2 = s;
  }
}
// out = trace of the lower g x g block of G ((K + g) x g): ||Out||^2 after
// ts_combine_gram
__global__ void k_gh_trace(const double* __restrict__ G, int K, int g, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int j = 0; j < g; ++j) s += G[K + j + (int64_t)(K + g) * j];
    *out = s;
  }
}

}  // namespace
}  // namespace bks

using namespace bks;

extern "C" void bks_gen_hooi_params_default(bks_gen_hooi_params* p) {
  if (!p) return;
  *p = bks_gen_hooi_params{};
  p->r1 = p->r2 = p->r3 = 2;
  p->tol = 1e-10;
  p->max_iter = 5000;
  p->grad_every = 10;
  p->seed = 1;
}

// HOOI for a general tensor (Section 6.1): U from the r1 leading left
// singular vectors of unfold_1(A.(V,W)_{2,3}), then V from
// unfold_2(A.(U,W)_{1,3}) with the new U, then W from unfold_3(A.(U,V)_{1,2})
// with the new U and V.  The G-gradient in global coordinates (three terms
// (I - Q Q^T) T F^T) every grad_every iterations, at the start of the
// iteration.  FP64.
extern "C" int bks_gen_hooi_solve(const bks_tensor* t, const bks_gen_hooi_params* prm,
                                  const double* U0, const double* V0, const double* W0,
                                  double* U, double* V, double* W, double* F, bks_info* info,
                                  void* stream) {
  if (!t || !prm) return fail(BKS_EINVAL, "null tensor or params");
  BKS_TRY(require_general(t));
  if (!U || !V || !W || !F) return fail(BKS_EINVAL, "null output");
  const int r[3] = {prm->r1, prm->r2, prm->r3};
  const int64_t d[3] = {t->l, t->m, t->n};
  for (int md = 0; md < 3; ++md) {
    if (r[md] < 1 || r[md] > 8) return fail(BKS_EUNSUPPORTED, "ranks must be in 1..8");
    if (r[md] > d[md]) return fail(BKS_EINVAL, "rank larger than the dimension");
  }
  const int w[3] = {r[1] * r[2], r[0] * r[2], r[0] * r[1]};
  for (int md = 0; md < 3; ++md)
    if (w[md] > kGenBlockMax) return fail(BKS_EUNSUPPORTED, "products of two ranks must be <= 32");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  DenseWork ws;
  DevBuf Qb[3], Tb[3], gout[3], G, FT, FF, sc;
  for (int md = 0; md < 3; ++md) {
    BKS_TRY(Qb[md].alloc(sizeof(double) * (size_t)d[md] * r[md], s));
    BKS_TRY(Tb[md].alloc(sizeof(double) * (size_t)d[md] * w[md], s));
    BKS_TRY(gout[md].alloc(sizeof(double) * (size_t)d[md] * r[md], s));
  }
  BKS_TRY(G.alloc(sizeof(double) * (kGenBlockMax + 8) * kGenBlockMax, s));
  BKS_TRY(FT.alloc(sizeof(double) * 3 * kGenBlockMax * 8, s));
  BKS_TRY(FF.alloc(sizeof(double) * 3 * 64, s));
  BKS_TRY(sc.alloc(sizeof(double) * 8, s));
  const double* starts[3] = {U0, V0, W0};
  for (int md = 0; md < 3; ++md) {
    if (starts[md]) BKS_TRY(gcopy2d(starts[md], d[md], d[md], r[md], Qb[md].as<double>(), d[md], s));
    else BKS_TRY(random_orthonormal(prm->seed, (uint64_t)(md + 1), d[md], r[md], Qb[md].as<double>(), ws, s));
  }
  double* Q[3] = {Qb[0].as<double>(), Qb[1].as<double>(), Qb[2].as<double>()};
  double* T[3] = {Tb[0].as<double>(), Tb[1].as<double>(), Tb[2].as<double>()};
  static const int oth[3][2] = {{1, 2}, {0, 2}, {0, 1}};
  auto contract = [&](int md) -> int {
    const int oa = oth[md][0], ob = oth[md][1];
    return gen_contract_x(t, md + 1, Q[oa], d[oa], r[oa], Q[ob], d[ob], r[ob], T[md], d[md], s);
  };
  const int every = std::max(1, prm->grad_every);
  int it = 0, hist_len = 0;
  double grad = INFINITY, nf = 0;
  bool converged = false;
  for (;; ++it) {
    BKS_TRY(contract(0));
    if (it % every == 0 || it >= prm->max_iter) {
      // the gradient at (U, V, W): T2, T3 at the same point
      BKS_TRY(contract(1));
      BKS_TRY(contract(2));
      BKS_CUDA_TRY(cudaMemsetAsync(sc.p, 0, sizeof(double) * 4, s));
      for (int md = 0; md < 3; ++md) {
        double* ft = FT.as<double>() + md * kGenBlockMax * 8;
        double* ff = FF.as<double>() + md * 64;
        BKS_TRY(ts_gram(Q[md], d[md], r[md], T[md], d[md], w[md], d[md], G.as<double>(), ws, s));
        k_gh_small<<<1, 128, 0, s>>>(G.as<double>(), r[md], w[md], ft, ff,
                                     md == 0 ? sc.as<double>() + 3 : nullptr); ::bks::note_launch();
        BKS_TRY(ts_combine_gram(Q[md], d[md], r[md], T[md], d[md], w[md], ff, ft, r[md],
                                gout[md].as<double>(), d[md], d[md], G.as<double>(), ws, s));
        k_gh_trace<<<1, 32, 0, s>>>(G.as<double>(), r[md], r[md], sc.as<double>() + md); ::bks::note_launch();
        BKS_CUDA_TRY(cudaGetLastError());
      }
      double h[4];
      BKS_CUDA_TRY(cudaMemcpyAsync(h, sc.p, sizeof(h), cudaMemcpyDeviceToHost, s));
      BKS_CUDA_TRY(cudaStreamSynchronize(s));
      grad = std::sqrt(std::max(0.0, h[0] + h[1] + h[2]));
      nf = std::sqrt(std::max(0.0, h[3]));
      const double rel = nf > 0 ? grad / nf : INFINITY;
      if (info && info->history && hist_len < info->history_cap) {
        info->history[2 * hist_len] = rel;
        info->history[2 * hist_len + 1] = nf;
        ++hist_len;
      }
      if (!std::isfinite(grad)) return fail(BKS_ENUMERIC, "NaN or Inf in the gradient");
      if (rel <= prm->tol) { converged = true; break; }
      if (it >= prm->max_iter) break;
    }
    // U from T1 (at V, W); V from T2 at the new U; W from T3 at the new U, V
    BKS_TRY(top_left_singular(T[0], d[0], d[0], w[0], r[0], Q[0], d[0], ws, s));
    BKS_TRY(contract(1));
    BKS_TRY(top_left_singular(T[1], d[1], d[1], w[1], r[1], Q[1], d[1], ws, s));
    BKS_TRY(contract(2));
    BKS_TRY(top_left_singular(T[2], d[2], d[2], w[2], r[2], Q[2], d[2], ws, s));
  }
  // F = U^T T1 at the evaluated point: FT of mode 1 holds F^T (w1 x r1)
  {
    const double* ft = FT.as<double>();
    // unfold_1(F) = (F^T)^T: r1 x w1, F[a + r1 (b + r2 c)]
    std::vector<double> h((size_t)w[0] * r[0]);
    BKS_CUDA_TRY(cudaMemcpyAsync(h.data(), ft, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<double> f(h.size());
    for (int a = 0; a < r[0]; ++a)
      for (int j = 0; j < w[0]; ++j) f[a + (size_t)r[0] * j] = h[j + (size_t)w[0] * a];
    BKS_CUDA_TRY(cudaMemcpyAsync(F, f.data(), sizeof(double) * f.size(), cudaMemcpyHostToDevice, s));
  }
  double* outs[3] = {U, V, W};
  for (int md = 0; md < 3; ++md) BKS_TRY(gcopy2d(Q[md], d[md], d[md], r[md], outs[md], d[md], s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = it;
    info->converged = converged ? 1 : 0;
    info->grad_rel = nf > 0 ? grad / nf : INFINITY;
    info->normF = nf;
    info->k1 = r[0];
    info->k2 = r[1];
    info->k3 = r[2];
    info->inner_sweeps = 0;
    info->fp32_iters = 0;
    info->history_len = hist_len;
    for (int q = 0; q < 5; ++q) info->phase_ms[q] = 0.0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!converged) return fail(BKS_ENOTCONV, "HOOI not converged within max_iter");
  return BKS_OK;
}

extern "C" void bks_gen_params_default(bks_gen_params* p) {
  if (!p) return;
  *p = bks_gen_params{};
  p->r1 = p->r2 = p->r3 = 2;
  p->stages = 2;
  p->block_p = 4;
  p->tol = 1e-10;
  p->max_outer = 500;
  p->max_inner = 1000;
  p->variant = BKS_VARIANT_BK;
  p->tol_scale_free = 0;
  p->seed = 1;
  p->drop_tol = 1e-14;
  p->inner_tol = 0.0;
  p->inner_schedule = BKS_INNER_PAPER;
}

extern "C" int bks_gen_solve(const bks_tensor* t, const bks_gen_params* prm, const double* U0,
                             const double* V0, const double* W0, double* U, double* V, double* W,
                             double* F, bks_info* info, void* stream) {
  BKS_TRY(check_gen_params(t, prm));
  if (!U || !V || !W || !F) return fail(BKS_EINVAL, "null output");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  GenState S;
  BKS_TRY(S.init(t, prm, s));
  const double* starts[3] = {U0, V0, W0};
  for (int md = 0; md < 3; ++md) {
    if (starts[md])
      BKS_TRY(gcopy2d(starts[md], S.dim[md], S.dim[md], S.r[md], S.Bp(md), S.dim[md], s));
    else
      BKS_TRY(random_orthonormal(prm->seed, (uint64_t)(md + 1), S.dim[md], S.r[md], S.Bp(md), S.ws, s));
  }
  int it = 0, hist_len = 0;
  double grad = 0, nf = 0;
  bool converged = false;
  int status = BKS_OK;
  for (;; ++it) {
    BKS_TRY(S.stage1(&grad, &nf));
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
    if (rel <= prm->tol) {
      converged = true;
      break;
    }
    if (it >= prm->max_outer) break;
    BKS_TRY(S.expand_rest());
    // inner tolerance on ||grad_C|| / ||F_C||: the outer one (Section 6.2),
    // or with BKS_INNER_FAST an inexact one a hundred times below the
    // current outer gradient and at least a tenth of the outer tolerance
    const double otol = prm->tol_scale_free ? prm->tol * nf : prm->tol;
    const bool fast = prm->inner_schedule == BKS_INNER_FAST;
    const double itol = prm->inner_tol > 0 ? prm->inner_tol
                        : fast ? std::max(0.1 * otol, 0.01 * (nf > 0 ? grad / nf : 0.0)) : otol;
    BKS_TRY(S.inner_and_restart(itol, fast ? 0 : kGenStartSweeps));
  }
  // outputs: the point whose gradient was evaluated last
  double* outs[3] = {U, V, W};
  for (int md = 0; md < 3; ++md)
    BKS_TRY(gcopy2d(S.Bp(md), S.dim[md], S.dim[md], S.r[md], outs[md], S.dim[md], s));
  BKS_TRY(gcopy2d(S.H1.as<double>(), S.r[0], S.r[0], S.r[1] * S.r[2], F, S.r[0], s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = it;
    info->converged = converged ? 1 : 0;
    info->grad_rel = nf > 0 ? (prm->tol_scale_free ? grad / (nf * nf) : grad / nf) : INFINITY;
    info->normF = nf;
    info->k1 = S.last_k[0] ? S.last_k[0] : S.k[0];
    info->k2 = S.last_k[1] ? S.last_k[1] : S.k[1];
    info->k3 = S.last_k[2] ? S.last_k[2] : S.k[2];
    info->inner_sweeps = S.inner_sweeps;
    info->fp32_iters = 0;
    info->history_len = hist_len;
    for (int q = 0; q < 5; ++q) info->phase_ms[q] = 0.0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status != BKS_OK) return status;
  if (!converged) return fail(BKS_ENOTCONV, "not converged within the iteration limits");
  return BKS_OK;
}
