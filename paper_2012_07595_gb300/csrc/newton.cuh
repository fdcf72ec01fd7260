// Newton-Grassmann step of the inner solve (newton.cu).
#pragma once
#include "common.cuh"

namespace bks {

constexpr int kNgMaxK = 128;  // k1, k3 <= 128
constexpr int kNgMaxR = 8;    // r1, r3 <= 8
constexpr int kNgSmemN = 224; // the FP32 factor of -H stays in shared memory up to N = 224

// Device workspace of the Newton steps, grown on demand, kept per thread
// and device with the inner-solve workspace.
struct NewtonWork {
  DevBuf Up, Wp, F0, B1, DUp, B3, G, B11, B13, S, S3, M1, M3, grad, z, res, w32, A, A32, flag;
  int ensure(int k1, int k3, int r1, int r3, cudaStream_t s);
};

// One Newton step from (Ug, Wg) (device, k1 x r1 and k3 x r3, orthonormal)
// given the contractions there: D = C x_3 Wg^T, T1 = unfold_1 C.(., Ug, Wg),
// E = C x_1 Ug^T, T3 = unfold_3 C.(Ug, Ug, .) in the cooperative inner
// kernel's layouts.  Writes the new point to Un, Wn; w.flag[0] = 1 when -H
// is not positive definite (then Un, Wn are not a step and must be
// discarded).  Stream-ordered; no host synchronisation.
int newton_step(const double* D, const double* T1, const double* E, const double* T3,
                const double* Ug, const double* Wg, int k1, int k3, int r1, int r3,
                double* Un, double* Wn, NewtonWork& w, cudaStream_t s);

}  // namespace bks
