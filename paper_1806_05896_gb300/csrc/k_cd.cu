// Convection-diffusion operator with SUPG (Section 5.2) as a stored 9-point stencil per
// node (assembled on every multigrid level with that level's mesh size).
//
// L = eps K + N + S on Q1 elements of the unit square:
//   K_e[a,b] = int grad phi_b . grad phi_a,     N_e[a,b] = int (w . grad phi_b) phi_a,
//   S_e[a,b] = delta_e int (w . grad phi_b)(w . grad phi_a),
//   delta_e  = h_e / (2|w_e|) (1 - 1/Pe_e) if Pe_e = |w_e| h_e / (2 eps) > 1, else 0,
// w_e the wind at the element centre, h_e the element length along w_e. The integrals use
// 3 Gauss points per direction, exact for the polynomial wind
// w = (2 y (1 - x^2), -2 x (1 - y^2)).
// coef[o * field + node] = L[node, node + off_o], off_o = (dy, dx) with o = (dy+1)*3 + (dx+1);
// entries at non-interior nodes are zero.
#include "kernels.h"

namespace {

IPM_D void wind(double x, double y, double& wx, double& wy) {
  wx = 2.0 * y * (1.0 - x * x);
  wy = -2.0 * x * (1.0 - y * y);
}

// element matrix of L for the element with lower-left node (ex, ey): Le[a][b], local
// index a = ax + 2 ay
IPM_D void element_matrix(double h, double eps, int ex, int ey, double Le[4][4]) {
  const double gp[3] = {0.5 - 0.5 * 0.7745966692414834, 0.5, 0.5 + 0.5 * 0.7745966692414834};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  const double x0 = ex * h, y0 = ey * h;
  double cwx, cwy;
  wind(x0 + 0.5 * h, y0 + 0.5 * h, cwx, cwy);
  const double wn = sqrt(cwx * cwx + cwy * cwy);
  const double wmax = fmax(fabs(cwx), fabs(cwy));
  const double he = wn > 0.0 ? h * wn / wmax : h;
  const double pe = wn * he / (2.0 * eps);
  const double delta = pe > 1.0 ? he / (2.0 * wn) * (1.0 - 1.0 / pe) : 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) Le[a][b] = 0.0;
  for (int qy = 0; qy < 3; ++qy)
    for (int qx = 0; qx < 3; ++qx) {
      const double s = gp[qx], t = gp[qy], wq = gw[qx] * gw[qy];
      double wx, wy;
      wind(x0 + h * s, y0 + h * t, wx, wy);
      double phi[4], dx[4], dy[4];  // values and physical gradients
      for (int a = 0; a < 4; ++a) {
        const int ax = a & 1, ay = a >> 1;
        const double fx = ax ? s : 1.0 - s, fy = ay ? t : 1.0 - t;
        const double gx = ax ? 1.0 : -1.0, gy = ay ? 1.0 : -1.0;
        phi[a] = fx * fy;
        dx[a] = gx * fy / h;
        dy[a] = fx * gy / h;
      }
      for (int a = 0; a < 4; ++a) {
        const double wga = wx * dx[a] + wy * dy[a];
        for (int b = 0; b < 4; ++b) {
          const double wgb = wx * dx[b] + wy * dy[b];
          const double k = dx[a] * dx[b] + dy[a] * dy[b];
          Le[a][b] += wq * h * h * (eps * k + wgb * phi[a] + delta * wgb * wga);
        }
      }
    }
}

__global__ void k_cd_coef(GridDesc g, double eps, double* __restrict__ coef) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  double acc[9];
  for (int o = 0; o < 9; ++o) acc[o] = 0.0;
  for (int e = 0; e < 4; ++e) {
    const int ex = i - 1 + (e & 1), ey = j - 1 + (e >> 1);
    double Le[4][4];
    element_matrix(g.h, eps, ex, ey, Le);
    const int a = (i - ex) + 2 * (j - ey);
    for (int b = 0; b < 4; ++b) {
      const int bx = ex + (b & 1), by = ey + (b >> 1);
      const int o = (by - j + 1) * 3 + (bx - i + 1);
      acc[o] += Le[a][b];
    }
  }
  for (int o = 0; o < 9; ++o) coef[(long long)o * g.field + c] = acc[o];
}

__global__ void k_to_float(long long n, const double* __restrict__ x, float* __restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (float)x[t];
}

}  // namespace

void launch_cd_coef(const GridDesc& g, double eps, double* coef, cudaStream_t s) {
  count_launches(1);
  k_cd_coef<<<interior_grid(g), interior_block(), 0, s>>>(g, eps, coef);
}

void launch_to_float(long long n, const double* x, float* y, cudaStream_t s) {
  count_launches(1);
  long long b = (n + 255) / 256;
  k_to_float<<<(int)(b < 4096 ? b : 4096), 256, 0, s>>>(n, x, y);
}
