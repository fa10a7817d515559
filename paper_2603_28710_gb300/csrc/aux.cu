// Auxiliary FP64 kernels: initial conditions at the nodes, conserved totals, maximum
// signal speed (for the CFL time step), L2 error against the exact vortex and a finiteness
// check.  Reductions are two-pass with a fixed block count and a fixed combination order,
// so their results do not depend on scheduling.
#include <math.h>

#include "adg_internal.h"

namespace adg {

namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ void node_coords(int dim, int N, int node, int* ix) {
  ix[0] = node % N;
  ix[1] = (node / N) % N;
  ix[2] = dim == 3 ? node / (N * N) : 0;
}

__device__ __forceinline__ void elem_coords_rt(const MeshArgs& m, int64_t e, int* c) {
  c[0] = (int)(e % m.n[0]);
  int64_t t = e / m.n[0];
  c[1] = (int)(t % m.n[1]);
  c[2] = (int)(t / m.n[1]);
}

struct VortexParams {
  double lo[3], h[3];
  double gamma, t, beta, x0, y0, Lx, Ly;
};

// Isentropic vortex of the 2D benchmark on the periodic box, nearest periodic image of the
// advected centre (x0 + t, y0); rho = (1 - (g-1) b^2 e^{2(1-r^2)} / (16 g pi^2))^{1/(g-1)},
// p = rho^g, u = 1 - b e^{1-r^2} dy / (2 pi), v = b e^{1-r^2} dx / (2 pi).
__device__ void vortex_state(int dim, const VortexParams& P, const double* x, double* w) {
  const double pi = 3.14159265358979323846;
  const double g = P.gamma;
  double dx = x[0] - (P.x0 + P.t);
  double dy = x[1] - P.y0;
  dx -= P.Lx * floor(dx / P.Lx + 0.5);
  dy -= P.Ly * floor(dy / P.Ly + 0.5);
  const double r2 = dx * dx + dy * dy;
  const double ex = exp(1.0 - r2);
  const double u = 1.0 - P.beta * ex * dy / (2.0 * pi);
  const double v = P.beta * ex * dx / (2.0 * pi);
  const double rho =
      pow(1.0 - (g - 1.0) / (16.0 * g * pi * pi) * P.beta * P.beta * ex * ex, 1.0 / (g - 1.0));
  const double p = pow(rho, g);
  w[0] = rho;
  w[1] = rho * u;
  w[2] = rho * v;
  if (dim == 3) w[3] = 0.0;
  w[dim + 1] = p / (g - 1.0) + 0.5 * rho * (u * u + v * v);
}

__global__ void init_vortex_kernel(int dim, int N, MeshArgs m, VortexParams P,
                                   const OpTables* tab, double* u) {
  int ND = dim == 3 ? N * N * N : N * N;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m.ne * ND) return;
  int64_t e = g / ND;
  int node = (int)(g - e * ND);
  int ix[3], ec[3];
  node_coords(dim, N, node, ix);
  elem_coords_rt(m, e, ec);
  double x[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) x[d] = P.lo[d] + (ec[d] + 0.5 * (tab->xi[ix[d]] + 1.0)) * P.h[d];
  double w[5];
  vortex_state(dim, P, x, w);
  for (int v = 0; v < dim + 2; ++v) u[((int64_t)v * m.ne + e) * ND + node] = w[v];
}

__global__ void init_tgv_kernel(int N, MeshArgs m, VortexParams P, double mach,
                                const OpTables* tab, double* u) {
  int ND = N * N * N;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m.ne * ND) return;
  int64_t e = g / ND;
  int node = (int)(g - e * ND);
  int ix[3], ec[3];
  node_coords(3, N, node, ix);
  elem_coords_rt(m, e, ec);
  double x[3];
  for (int d = 0; d < 3; ++d) x[d] = P.lo[d] + (ec[d] + 0.5 * (tab->xi[ix[d]] + 1.0)) * P.h[d];
  const double g0 = P.gamma;
  const double p0 = 1.0 / (g0 * mach * mach);
  const double ux = sin(x[0]) * cos(x[1]) * cos(x[2]);
  const double uy = -cos(x[0]) * sin(x[1]) * cos(x[2]);
  const double p = p0 + (cos(2.0 * x[0]) + cos(2.0 * x[1])) * (cos(2.0 * x[2]) + 2.0) / 16.0;
  const double rho = p / p0;
  double w[5] = {rho, rho * ux, rho * uy, 0.0, p / (g0 - 1.0) + 0.5 * rho * (ux * ux + uy * uy)};
  for (int v = 0; v < 5; ++v) u[((int64_t)v * m.ne + e) * ND + node] = w[v];
}

// Fixed-order block reduction of kRedThreads values (sum or max).
template <bool MAX>
__device__ double block_reduce(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double a = sh[threadIdx.x], b = sh[threadIdx.x + s];
      sh[threadIdx.x] = MAX ? fmax(a, b) : a + b;
    }
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// partial[blk][v] = sum over the block's nodes of omega_q |J| u_v
__global__ void conservation_kernel(int dim, int N, MeshArgs m, const OpTables* tab, double J,
                                    const double* u, double* partial) {
  __shared__ double sh[kRedThreads];
  int ND = dim == 3 ? N * N * N : N * N;
  int64_t total = m.ne * ND;
  int64_t chunk = (total + gridDim.x - 1) / gridDim.x;
  int64_t beg = chunk * blockIdx.x, end = beg + chunk < total ? beg + chunk : total;
  for (int v = 0; v < dim + 2; ++v) {
    double s = 0.0;
    for (int64_t g = beg + threadIdx.x; g < end; g += kRedThreads) {
      int64_t e = g / ND;
      int node = (int)(g - e * ND);
      int ix[3];
      node_coords(dim, N, node, ix);
      double wq = J;
      for (int d = 0; d < dim; ++d) wq *= tab->wq[ix[d]];
      s += wq * u[((int64_t)v * m.ne + e) * ND + node];
    }
    double r = block_reduce<false>(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x * 5 + v] = r;
  }
}

template <bool MAX>
__global__ void finish_kernel(int nv, int nblocks, const double* partial, double* out) {
  __shared__ double sh[kRedThreads];
  for (int v = 0; v < nv; ++v) {
    double s = MAX ? 0.0 : 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kRedThreads) {
      double x = partial[b * 5 + v];
      s = MAX ? fmax(s, x) : s + x;
    }
    double r = block_reduce<MAX>(s, sh);
    if (threadIdx.x == 0) out[v] = r;
  }
}

// max over nodes of |u| + c
__global__ void max_speed_kernel(int dim, int N, MeshArgs m, double gamma, const double* u,
                                 double* partial) {
  __shared__ double sh[kRedThreads];
  int ND = dim == 3 ? N * N * N : N * N;
  int64_t total = m.ne * ND;
  int64_t chunk = (total + gridDim.x - 1) / gridDim.x;
  int64_t beg = chunk * blockIdx.x, end = beg + chunk < total ? beg + chunk : total;
  double smax = 0.0;
  for (int64_t g = beg + threadIdx.x; g < end; g += kRedThreads) {
    int64_t e = g / ND;
    int node = (int)(g - e * ND);
    double w[5];
    for (int v = 0; v < dim + 2; ++v) w[v] = u[((int64_t)v * m.ne + e) * ND + node];
    double u2 = 0.0, kin = 0.0;
    for (int d = 0; d < dim; ++d) {
      double ud = w[1 + d] / w[0];
      u2 += ud * ud;
      kin += w[1 + d] * ud;
    }
    double p = (gamma - 1.0) * (w[dim + 1] - 0.5 * kin);
    double s = sqrt(u2) + sqrt(gamma * p / w[0]);
    smax = fmax(smax, s);
  }
  double r = block_reduce<true>(smax, sh);
  if (threadIdx.x == 0) partial[blockIdx.x * 5] = r;
}

// partial[blk][0..2] = squared L2 error contributions (density, momentum, energy)
__global__ void l2_vortex_kernel(int dim, int N, MeshArgs m, VortexParams P, const OpTables* tab,
                                 double J, const double* u, double* partial) {
  __shared__ double sh[kRedThreads];
  const int M = N + 1;
  const int ND = dim == 3 ? N * N * N : N * N;
  const int NP = dim == 3 ? M * M * M : M * M;
  int64_t total = m.ne * NP;
  int64_t chunk = (total + gridDim.x - 1) / gridDim.x;
  int64_t beg = chunk * blockIdx.x, end = beg + chunk < total ? beg + chunk : total;
  double acc[3] = {0, 0, 0};
  for (int64_t g = beg + threadIdx.x; g < end; g += kRedThreads) {
    int64_t e = g / NP;
    int pt = (int)(g - e * NP);
    int ip[3] = {pt % M, (pt / M) % M, dim == 3 ? pt / (M * M) : 0};
    int ec[3];
    elem_coords_rt(m, e, ec);
    double x[3] = {0, 0, 0}, wt = J;
    for (int d = 0; d < dim; ++d) {
      x[d] = P.lo[d] + (ec[d] + 0.5 * (tab->xe[ip[d]] + 1.0)) * P.h[d];
      wt *= tab->we[ip[d]];
    }
    double wex[5], wh[5];
    vortex_state(dim, P, x, wex);
    for (int v = 0; v < dim + 2; ++v) {
      double s = 0.0;
      for (int j = 0; j < ND; ++j) {
        int ix[3];
        node_coords(dim, N, j, ix);
        double phi = 1.0;
        for (int d = 0; d < dim; ++d) phi *= tab->Le[ip[d] * N + ix[d]];
        s += u[((int64_t)v * m.ne + e) * ND + j] * phi;
      }
      wh[v] = s;
    }
    double dr = wh[0] - wex[0], de = wh[dim + 1] - wex[dim + 1], dm = 0.0;
    for (int d = 0; d < dim; ++d) dm += (wh[1 + d] - wex[1 + d]) * (wh[1 + d] - wex[1 + d]);
    acc[0] += wt * dr * dr;
    acc[1] += wt * dm;
    acc[2] += wt * de * de;
  }
  for (int i = 0; i < 3; ++i) {
    double r = block_reduce<false>(acc[i], sh);
    if (threadIdx.x == 0) partial[blockIdx.x * 5 + i] = r;
  }
}

__global__ void check_finite_kernel(int64_t n, const double* u, int* flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int bad = 0;
  for (; i < n; i += stride) bad |= !isfinite(u[i]);
  if (bad) atomicOr(flag, 1);
}

VortexParams make_params(const double* lo, const double* h, double gamma, double t, double beta,
                         double x0, double y0, double Lx, double Ly) {
  VortexParams P;
  for (int d = 0; d < 3; ++d) {
    P.lo[d] = lo[d];
    P.h[d] = h[d];
  }
  P.gamma = gamma;
  P.t = t;
  P.beta = beta;
  P.x0 = x0;
  P.y0 = y0;
  P.Lx = Lx;
  P.Ly = Ly;
  return P;
}

unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_init_vortex(int dim, int N, const MeshArgs& m, const double* lo,
                               const double* h, const OpTables* tab, double gamma, double t,
                               double beta, double x0, double y0, double Lx, double Ly,
                               double* u, cudaStream_t s) {
  int ND = dim == 3 ? N * N * N : N * N;
  VortexParams P = make_params(lo, h, gamma, t, beta, x0, y0, Lx, Ly);
  init_vortex_kernel<<<grid_for(m.ne * ND, 256), 256, 0, s>>>(dim, N, m, P, tab, u);
  return cudaGetLastError();
}

cudaError_t launch_init_tgv(int N, const MeshArgs& m, const double* lo, const double* h,
                            const OpTables* tab, double gamma, double mach, double* u,
                            cudaStream_t s) {
  VortexParams P = make_params(lo, h, gamma, 0, 0, 0, 0, 1, 1);
  init_tgv_kernel<<<grid_for(m.ne * N * N * N, 256), 256, 0, s>>>(N, m, P, mach, tab, u);
  return cudaGetLastError();
}

cudaError_t launch_conservation(int dim, int N, const MeshArgs& m, const OpTables* tab,
                                double J, const double* u, double* partial, double* out,
                                int nblocks, cudaStream_t s) {
  conservation_kernel<<<nblocks, kRedThreads, 0, s>>>(dim, N, m, tab, J, u, partial);
  finish_kernel<false><<<1, kRedThreads, 0, s>>>(dim + 2, nblocks, partial, out);
  return cudaGetLastError();
}

cudaError_t launch_max_speed(int dim, int N, const MeshArgs& m, double gamma, const double* u,
                             double* partial, double* out, int nblocks, cudaStream_t s) {
  max_speed_kernel<<<nblocks, kRedThreads, 0, s>>>(dim, N, m, gamma, u, partial);
  finish_kernel<true><<<1, kRedThreads, 0, s>>>(1, nblocks, partial, out);
  return cudaGetLastError();
}

cudaError_t launch_l2_vortex(int dim, int N, const MeshArgs& m, const double* lo,
                             const double* h, const OpTables* tab, double gamma, double t,
                             double beta, double x0, double y0, double Lx, double Ly,
                             const double* u, double* partial, double* out, int nblocks,
                             cudaStream_t s) {
  VortexParams P = make_params(lo, h, gamma, t, beta, x0, y0, Lx, Ly);
  double J = 1.0;
  for (int d = 0; d < dim; ++d) J *= h[d] / 2.0;
  l2_vortex_kernel<<<nblocks, kRedThreads, 0, s>>>(dim, N, m, P, tab, J, u, partial);
  finish_kernel<false><<<1, kRedThreads, 0, s>>>(3, nblocks, partial, out);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(int64_t n, const double* u, int* flag, cudaStream_t s) {
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  check_finite_kernel<<<152 * 8, 256, 0, s>>>(n, u, flag);
  return cudaGetLastError();
}

}  // namespace adg
