// Autotuner of the contraction work tiles: for a stored tensor, time the
// mode-1 and triangle mode-3 contractions (FP32, widths 4 x 4) under a few
// (tile, split) plans and keep the fastest.  Power-law tensors differ in how
// their entries spread over rows, and the best cuts between "rows on one
// lane", "rows on one warp" and "rows split into pieces" depend on that
// spread.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace bks {

namespace {

int rebuild(bks_tensor* t, int tile, int split, cudaStream_t s) {
  t->m1.tile = t->m3.tile = tile;
  t->m1.split = t->m3.split = split;
  BKS_TRY(build_tile_plan(t->m1, t->nnz, s));
  BKS_TRY(build_tile_plan(t->m3, t->nnz, s));
  return BKS_OK;
}

}  // namespace

int autotune_tensor(bks_tensor* t, cudaStream_t s, int* tile_out, int* split_out) {
  static const int cand[][2] = {{8, 512}, {16, 512}, {64, 1024}, {128, 2048}, {32, 512}};
  const int p = 4;
  DevBuf X, Y, out;
  BKS_TRY(X.alloc(sizeof(float) * (size_t)t->m * p, s));
  BKS_TRY(Y.alloc(sizeof(float) * (size_t)t->n * p, s));
  const size_t outn = std::max<size_t>((size_t)t->m * p * p, (size_t)t->n * p * (p + 1) / 2);
  BKS_TRY(out.alloc(sizeof(float) * outn, s));
  BKS_CUDA_TRY(cudaMemsetAsync(X.p, 0, X.bytes, s));
  BKS_CUDA_TRY(cudaMemsetAsync(Y.p, 0, Y.bytes, s));
  cudaEvent_t e0, e1;
  BKS_CUDA_TRY(cudaEventCreate(&e0));
  BKS_CUDA_TRY(cudaEventCreate(&e1));
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } guard{e0, e1};
  float best = 1e30f;
  int bi = 1;
  for (int c = 0; c < (int)(sizeof(cand) / sizeof(cand[0])); ++c) {
    BKS_TRY(rebuild(t, cand[c][0], cand[c][1], s));
    float tot = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
      BKS_CUDA_TRY(cudaEventRecord(e0, s));
      BKS_TRY(contract_mode1(t, X.p, t->m, p, Y.p, t->n, p, out.p, t->m, BKS_F32, s));
      BKS_TRY(contract_mode3(t, X.p, t->m, p, nullptr, t->m, p, out.p, t->n, BKS_F32, s));
      BKS_CUDA_TRY(cudaEventRecord(e1, s));
      BKS_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      BKS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) tot += ms;  // first run warms the caches
    }
    if (tot < best) {
      best = tot;
      bi = c;
    }
  }
  if (bi != (int)(sizeof(cand) / sizeof(cand[0])) - 1) BKS_TRY(rebuild(t, cand[bi][0], cand[bi][1], s));
  if (tile_out) *tile_out = cand[bi][0];
  if (split_out) *split_out = cand[bi][1];
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  return BKS_OK;
}

int set_tiles(bks_tensor* t, int tile, int split, cudaStream_t s) {
  if (tile < 1 || split < kMinSplit || tile > kMaxTile || split > kMaxSplit)
    return fail(BKS_EINVAL, "tile must be in [1, 128] and split in [128, 4096]");
  if (t->m1.tile == tile && t->m1.split == split) return BKS_OK;
  BKS_TRY(rebuild(t, tile, split, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  return BKS_OK;
}

}  // namespace bks

extern "C" int bks_tensor_autotune(bks_tensor* t, int* tile, int* split, void* stream) {
  if (!t) return bks::fail(BKS_EINVAL, "null tensor");
  BKS_TRY(bks::require_symmetric(t));
  return bks::autotune_tensor(t, (cudaStream_t)stream, tile, split);
}

extern "C" int bks_tensor_set_tiles(bks_tensor* t, int tile, int split, void* stream) {
  if (!t) return bks::fail(BKS_EINVAL, "null tensor");
  BKS_TRY(bks::require_symmetric(t));
  return bks::set_tiles(t, tile, split, (cudaStream_t)stream);
}
