// Learned ghost-trace predictor in the solver: trace logging at subdomain faces (training
// data from synchronous runs), the training-sample builder, and the learned correction of
// the AT trace extrapolation at delayed subdomain faces.
//
// Per scalar channel (one variable, one side, one face node) with stored levels a0, a1, a2
// (newest first) and stage delay k_m = k + c_m, the AT extrapolation is
// E3 = sum_l c_l(k_m) a_l (Eq. 14 on traces, N_p = 2) and the linear one is
// E2 = a0 + k_m (a0 - a1); their difference e = E3 - E2 estimates the AT error scale.  The
// network sees x = ((a0 - a1)/s, (a1 - a2)/s, k/8, c_m) with s = |a0 - a1| + |a1 - a2| and
// predicts y ~ (truth - E3)/e, a learned next-order step; the corrected trace is E3 + e y,
// accepted only when y is finite and |y| <= trust, so no correction exceeds trust times
// AT's own error estimate.  Where e is at rounding level (|e| <= 1e-9 (|a0|+|a1|+|a2|)) AT
// stands.  Both sides of a face are corrected by the same rule from the same stored data,
// so the two neighbours still share one flux.
#include "kernels.cuh"

namespace adg {

cudaError_t mlp_infer(const uint16_t* params, const float* x, int64_t n, float* y, cudaStream_t s);

__device__ __forceinline__ bool learned_features(double a0, double a1, double a2, int k,
                                                 double cm, float* x, double* e_out) {
  const double km = k + cm;
  const double e3 = 0.5 * (km + 1.0) * (km + 2.0) * a0 - km * (km + 2.0) * a1 +
                    0.5 * km * (km + 1.0) * a2;
  const double e2 = a0 + km * (a0 - a1);
  const double e = e3 - e2;
  const double s = fabs(a0 - a1) + fabs(a1 - a2);
  *e_out = 0.0;
  // an error estimate at rounding level: AT is exact there already
  if (!(fabs(e) > 1e-9 * (fabs(a0) + fabs(a1) + fabs(a2)) && s > 1e-300)) return false;
  *e_out = e;
  const double inv = 1.0 / s;
  x[0] = (float)((a0 - a1) * inv);
  x[1] = (float)((a1 - a2) * inv);
  x[2] = 0.125f * (float)k;
  x[3] = (float)cm;
  return true;
}

namespace {

// Channel index of (slot, face node, side, var): ((slot * NF + j) * 2 + side) * NV + v.

// Pass 1, thread per (subdomain face, face node): AT extrapolation E of every channel of
// both sides, the level spread s and the network input x (x = 0, s = 0 where no
// correction applies: fresh data or constant levels).
template <int D, int N, typename R>
__global__ void __launch_bounds__(128) learned_features_kernel(const LearnArgs A) {
  using S = typename Arith<R>::S;
  constexpr int NF = IPow<N, D - 1>::value, NV = D + 2;
  const int npe = (int)A.npe;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npe * NF) return;
  const int slot = g / NF, j = g - slot * NF;
  int kt = A.uniform_delay;
  if (A.random) {
    const uint64_t ctr = (uint64_t)A.step * (uint64_t)A.n_iface + (uint64_t)A.pe_iface[slot];
    kt = (int)(splitmix64_dev(A.seed ^ ctr) % (uint64_t)(A.dmax + 1));
    if (A.step - (kt + 2) < 0) kt = 0;
  }
  S* Eout = reinterpret_cast<S*>(A.E);
  if (kt == 0) {
#pragma unroll
    for (int c = 0; c < 2 * NV; ++c) {
      A.s[g * 2 * NV + c] = 0.0;
      reinterpret_cast<float4*>(A.x)[g * 2 * NV + c] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return;
  }
  const int off = A.random ? kt : 0;
  const S* ring = reinterpret_cast<const S*>(A.ring);
  const int lvl_stride = 2 * NV * npe * NF;
  int lv[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    int q = (A.head - off - l) % A.depth;
    lv[l] = q < 0 ? q + A.depth : q;
  }
  const double cm = A.km[kt] - kt;  // stage offset c_m
#pragma unroll
  for (int side = 0; side < 2; ++side) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      R a[3];
      typename Arith<R>::Acc acc = acc_zero(typename Arith<R>::Acc());
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        a[l] = Arith<R>::load(ring + lv[l] * lvl_stride + ((side * NV + v) * npe + slot) * NF + j);
        acc = acc_fma(Arith<R>::pair(A.ctab[kt][l], A.ctabf[kt][l]), a[l], acc);
      }
      const int c = g * 2 * NV + side * NV + v;
      Arith<R>::store(Eout + c, acc_result(acc));
      float x[4];
      double s;
      const bool good = learned_features(Arith<R>::to_double(a[0]), Arith<R>::to_double(a[1]),
                                         Arith<R>::to_double(a[2]), kt, cm, x, &s);
      A.s[c] = good ? s : 0.0;
      reinterpret_cast<float4*>(A.x)[c] =
          good ? make_float4(x[0], x[1], x[2], x[3]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// Pass 3 (after the network evaluated y for every channel), thread per (face, face node):
// corrected traces (the trust test keeps E when y is not finite, |y| > trust or s = 0), then
// the Rusanov flux of Eq. 8 overwrites the face flux.
template <int D, int N, typename R>
__global__ void __launch_bounds__(128) learned_apply_kernel(const LearnArgs A) {
  using S = typename Arith<R>::S;
  constexpr int NF = IPow<N, D - 1>::value, NV = D + 2;
  const int npe = (int)A.npe;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npe * NF) return;
  const int slot = g / NF, j = g - slot * NF;
  // faces without a usable correction (fresh data, or constant levels everywhere) keep the
  // AT value the flux kernel wrote
  bool any = false;
#pragma unroll
  for (int c = 0; c < 2 * NV; ++c) any |= A.s[g * 2 * NV + c] != 0.0;
  if (!any) return;
  const S* Ein = reinterpret_cast<const S*>(A.E);
  R tr[2][NV];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int c = g * 2 * NV + side * NV + v;
      const R E = Arith<R>::load(Ein + c);
      const double s = A.s[c];
      const float y = A.y[c];
      tr[side][v] = (s != 0.0 && isfinite(y) && fabsf(y) <= A.trust)
                        ? E + Arith<R>::from_double(s * (double)y) : E;
    }
  }
  const int d = A.face_d[slot], e = A.face_e[slot];
  R f[NV];
  llf_flux<D, R>(tr[0], tr[1], d, Arith<R>::pair(A.gamma, A.gammaf), Arith<R>::pair(A.gm1, A.gm1f), f);
  S* fl = reinterpret_cast<S*>(A.fl);
  const int ne = (int)A.m.ne;
#pragma unroll
  for (int v = 0; v < NV; ++v) Arith<R>::store(fl + ((d * NV + v) * ne + e) * NF + j, f[v]);
}

// thread per (side, var, slot, face node): PE-face traces of the current stage input
template <int D, int N, typename R>
__global__ void log_kernel(const typename Arith<R>::S* tr, const int32_t* face_d,
                           const int32_t* face_e, MeshArgs m, int npe, double* out) {
  constexpr int NF = IPow<N, D - 1>::value, NV = D + 2;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 2 * NV * npe * NF) return;
  const int j = g % NF;
  const int slot = (g / NF) % npe;
  const int v = (g / (NF * npe)) % NV;
  const int side = g / (NF * npe * NV);
  const int d = face_d[slot], e = face_e[slot];
  int ec[3];
  elem_coords(m, e, ec);
  const int eh = elem_shift(m, e, ec, d, +1);
  const int ne = (int)m.ne;
  // side 0: high-side trace of e (minus state), side 1: low-side trace of its neighbour
  const int idx = side == 0 ? (((d * 2 + 1) * NV + v) * ne + e) * NF + j
                            : (((d * 2 + 0) * NV + v) * ne + eh) * NF + j;
  out[g] = Arith<R>::to_double(Arith<R>::load(tr + idx));
}

template <typename R>
struct LearnDispatch {
  template <int D, int N>
  static cudaError_t learn(const LearnArgs& a, cudaStream_t s) {
    constexpr int NF = IPow<N, D - 1>::value;
    const int64_t total = a.npe * NF;
    if (total == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 127) / 128);
    learned_features_kernel<D, N, R><<<blocks, 128, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = mlp_infer(a.mlp, reinterpret_cast<const float*>(a.x), total * 2 * (D + 2), a.y, s);
    if (e != cudaSuccess) return e;
    learned_apply_kernel<D, N, R><<<blocks, 128, 0, s>>>(a);
    return cudaGetLastError();
  }
  template <int D, int N>
  static cudaError_t log(const void* tr, const int32_t* fd, const int32_t* fe, const MeshArgs& m,
                         int64_t npe, double* out, cudaStream_t s) {
    constexpr int NF = IPow<N, D - 1>::value;
    const int64_t total = 2 * (D + 2) * npe * NF;
    if (total == 0) return cudaSuccess;
    log_kernel<D, N, R><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const typename Arith<R>::S*>(tr), fd, fe, m, (int)npe, out);
    return cudaGetLastError();
  }
};


template <typename R>
cudaError_t learn_r(int dim, int N, const LearnArgs& a, cudaStream_t s) {
#define CALL_L(D_, N_) LearnDispatch<R>::template learn<D_, N_>(a, s)
  if (dim == 2) {
    switch (N) {
      case 2: return CALL_L(2, 2);
      case 3: return CALL_L(2, 3);
      case 4: return CALL_L(2, 4);
      case 5: return CALL_L(2, 5);
      case 6: return CALL_L(2, 6);
      case 7: return CALL_L(2, 7);
      case 8: return CALL_L(2, 8);
    }
  } else if (dim == 3) {
    switch (N) {
      case 2: return CALL_L(3, 2);
      case 3: return CALL_L(3, 3);
      case 4: return CALL_L(3, 4);
      case 5: return CALL_L(3, 5);
      case 6: return CALL_L(3, 6);
    }
  }
#undef CALL_L
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t log_r(int dim, int N, const void* tr, const int32_t* fd, const int32_t* fe,
                  const MeshArgs& m, int64_t npe, double* out, cudaStream_t s) {
#define CALL_G(D_, N_) LearnDispatch<R>::template log<D_, N_>(tr, fd, fe, m, npe, out, s)
  if (dim == 2) {
    switch (N) {
      case 2: return CALL_G(2, 2);
      case 3: return CALL_G(2, 3);
      case 4: return CALL_G(2, 4);
      case 5: return CALL_G(2, 5);
      case 6: return CALL_G(2, 6);
      case 7: return CALL_G(2, 7);
      case 8: return CALL_G(2, 8);
    }
  } else if (dim == 3) {
    switch (N) {
      case 2: return CALL_G(3, 2);
      case 3: return CALL_G(3, 3);
      case 4: return CALL_G(3, 4);
      case 5: return CALL_G(3, 5);
      case 6: return CALL_G(3, 6);
    }
  }
#undef CALL_G
  return cudaErrorInvalidValue;
}

// training samples: picks[n] = (channel, step, stage, delay) into a trace log of records
// [step * stages + stage][channel]; levels are stage-0 records of steps n-k, n-k-1, n-k-2
__global__ void samples_kernel(const double* log, int64_t rec_len, int stages,
                               const int32_t* picks, int n, const double* ctab /*[k][m][3]*/,
                               const double* kmtab /*[k][m]*/, int kmax, float* x, float* target,
                               int* ok) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t c = picks[4 * i], step = picks[4 * i + 1];
  const int m = picks[4 * i + 2], k = picks[4 * i + 3];
  double a[3];
  for (int l = 0; l < 3; ++l) a[l] = log[((step - k - l) * stages) * rec_len + c];
  const double truth = log[(step * stages + m) * rec_len + c];
  const double* cc = ctab + ((k * stages) + m) * 3;
  const double E = cc[0] * a[0] + cc[1] * a[1] + cc[2] * a[2];
  double s;
  float xi[4];
  const bool good = learned_features(a[0], a[1], a[2], k, kmtab[k * stages + m] - k, xi, &s);
  for (int q = 0; q < 4; ++q) x[4 * i + q] = good ? xi[q] : 0.0f;
  target[i] = good ? (float)((truth - E) / s) : 0.0f;
  ok[i] = good ? 1 : 0;
  (void)kmax;
}

}  // namespace

cudaError_t launch_learned(int prec, int dim, int N, const LearnArgs& a, cudaStream_t s) {
  switch (prec) {
    case 0: return learn_r<double>(dim, N, a, s);
    case 1: return learn_r<float>(dim, N, a, s);
    case 2: return learn_r<df64>(dim, N, a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_log_traces(int prec, int dim, int N, const void* tr, const int32_t* fd,
                              const int32_t* fe, const MeshArgs& m, int64_t npe, double* out,
                              cudaStream_t s) {
  switch (prec) {
    case 0: return log_r<double>(dim, N, tr, fd, fe, m, npe, out, s);
    case 1: return log_r<float>(dim, N, tr, fd, fe, m, npe, out, s);
    case 2: return log_r<df64>(dim, N, tr, fd, fe, m, npe, out, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_samples(const double* log, int64_t rec_len, int stages, const int32_t* picks,
                           int n, const double* ctab, const double* kmtab, int kmax, float* x,
                           float* target, int* ok, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  samples_kernel<<<(n + 255) / 256, 256, 0, s>>>(log, rec_len, stages, picks, n, ctab, kmtab, kmax,
                                                 x, target, ok);
  return cudaGetLastError();
}

}  // namespace adg
