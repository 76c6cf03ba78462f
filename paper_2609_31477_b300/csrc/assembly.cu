// Element kernels of the ALE Navier-Stokes / pseudo-solid / multiplier system.
//
// Residual (Eq. nonlinear_functional_discrete), per 9-node quad and 3x3 Gauss
// points, with u_dot_a = c0 u_a + hu_a and w_a = c0 x_a + hx_a (nodal BDF rates):
//   R[u_a,i] = int_Ot N_a rho (u_dot + ((u-w).grad)u)_i + grad N_a . sigma_i,
//              sigma = -p I + mu (grad u + grad u^T)
//   R[p_c]   = -int_Ot M_c div u
//   R[x_a,i] = int_O0 lame (grad_X N_a)_i (div_X x - 2) + 2 lame grad_X N_a . eps_i,
//              eps = sym(grad_X x) - I
// Gamma edges: R[u_b,i] -= int N_b lambda_i ds, R[lambda_b,i] = -int N_b (u-w)_i ds,
// border rows R[delta_i] = k delta_i + int_Gamma lambda_i ds.
//
// Jacobian: the analytic derivative of these integrals (Section 3.2), including
// the shape derivatives with respect to x: with G = grad_x(dx) for dx = N_b e_k,
// d(det J) = det J g_b,k, d(g_a,j) = -g_a,k g_b,j, d(L_ij) = -L_ik g_b,j and
// d(w) = c0 N_b e_k.  Position columns of Gamma nodes are the delta columns
// (x = X + delta on Gamma).
//
// One thread computes one element row (all of its columns), so every CSR slot
// of an element, including the merged delta columns, is written by one
// thread; elements of one colour share no node, so one colour per launch
// needs no atomics and the sums are deterministic.
#include <cuda_runtime.h>

#include "viv_internal.h"

namespace viv {
namespace {

constexpr int EPB = 8;              // elements per block
constexpr int ROWS = 40;            // element rows: 18 u, 4 p, 18 x
constexpr int ASM_THREADS = EPB * ROWS;
constexpr int QP_DATA = 59;         // per quadrature point values kept in shared memory

__device__ __forceinline__ void lag2(double s, double* L, double* dL) {
  L[0] = (1 - s) * (1 - 2 * s);
  L[1] = 4 * s * (1 - s);
  L[2] = s * (2 * s - 1);
  dL[0] = 4 * s - 3;
  dL[1] = 4 - 8 * s;
  dL[2] = 4 * s - 1;
}

__device__ __constant__ double c_gpt[3] = {0.11270166537925831148, 0.5, 0.88729833462074168852};
__device__ __constant__ double c_gwt[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};

template <class T>
struct Tables {
  T N[9][9];       // [qp][node]
  T dN[9][9][2];
  T M[9][4];
  T W[9];
};

template <class T>
__device__ void build_tables(Tables<T>& tb) {
  for (int t = threadIdx.x; t < 81; t += blockDim.x) {
    int q = t / 9, nd = t % 9;
    int i = q % 3, j = q / 3, a = nd % 3, b = nd / 3;
    double Li[3], dLi[3], Lj[3], dLj[3];
    lag2(c_gpt[i], Li, dLi);
    lag2(c_gpt[j], Lj, dLj);
    tb.N[q][nd] = (T)(Li[a] * Lj[b]);
    tb.dN[q][nd][0] = (T)(dLi[a] * Lj[b]);
    tb.dN[q][nd][1] = (T)(Li[a] * dLj[b]);
    if (nd < 4) {
      int c = nd % 2, dd = nd / 2;
      double li = c ? c_gpt[i] : 1 - c_gpt[i];
      double lj = dd ? c_gpt[j] : 1 - c_gpt[j];
      tb.M[q][nd] = (T)(li * lj);
    }
    if (nd == 0) tb.W[q] = (T)(c_gwt[i] * c_gwt[j]);
  }
}

// per element node data in shared memory
template <class T>
struct ElemNodes {
  T X[9][2], x[9][2], u[9][2], ud[9][2], wn[9][2], p[4];
  T lame;
};

// qp data layout (offsets into a QP_DATA-sized record)
enum {
  Q_WDET = 0, Q_G = 1, Q_UW = 19, Q_L = 21, Q_SIG = 25, Q_INERT = 28, Q_DIV = 30,
  Q_WDET0 = 31, Q_G0 = 32, Q_EPS = 50, Q_TR = 53,
  Q_FU = 54, Q_GP = 56, Q_FX = 57   // manufactured source terms (zero unless enabled)
};

// Manufactured source of the steady 2-D test (Section 5.1's velocity and
// pressure without their time factors, on a mesh deformed by
// chi(X) = X + amp sin(pi X) sin(pi Y) (1, 1), lambda_s = mu_s = 1):
//   f_u = rho (u.grad) u + grad p - mu (lap u + grad div u)   at x = chi(X_q)
//   g_p = div u                                               at x = chi(X_q)
//   f_x = -div_X sigma_s(chi) = amp (4 pi^2 s - 2 pi^2 cos pi X cos pi Y) (1, 1)
__device__ __noinline__ void mms_source(double X, double Y, double amp, double rho, double mu, double* fu, double* gp,
                           double* fx) {
  const double pi = 3.14159265358979323846;
  const double s = sin(pi * X) * sin(pi * Y);
  const double x = X + amp * s, y = Y + amp * s;
  const double sx = sin(pi * x), cx = cos(pi * x), sy = sin(pi * y), cy = cos(pi * y);
  const double u1 = sx * cy, u2 = sx * sy;
  const double u1x = pi * cx * cy, u1y = -pi * sx * sy, u2x = pi * cx * sy, u2y = pi * sx * cy;
  const double lap1 = -2 * pi * pi * sx * cy, lap2 = -2 * pi * pi * sx * sy;
  const double gd1 = -pi * pi * sx * cy + pi * pi * cx * cy, gd2 = -pi * pi * cx * sy - pi * pi * sx * sy;
  const double px = -pi * sx * cy, py = -pi * cx * sy;
  fu[0] = rho * (u1 * u1x + u2 * u1y) + px - mu * (lap1 + gd1);
  fu[1] = rho * (u1 * u2x + u2 * u2y) + py - mu * (lap2 + gd2);
  *gp = u1x + u2y;
  const double f = amp * (4 * pi * pi * s - 2 * pi * pi * cos(pi * X) * cos(pi * Y));
  fx[0] = f;
  fx[1] = f;
}

// Manufactured source of the time-dependent 2-D test (Section 5.1's fields
// with their time factors, u = t^3 U, p = t^2 P with U, P the steady fields
// above, on a mesh moved by chi(X, t) = X + amp sin(pi t) sin(pi X) sin(pi Y) (1, 1),
// lambda_s = mu_s = 1):
//   f_u = rho (d_t u + (u.grad) u) + grad p - mu (lap u + grad div u)
//       = rho (3 t^2 U + t^6 (U.grad) U) + t^2 grad P - mu t^3 (lap U + grad div U)
//   g_p = t^3 div U,  f_x = sin(pi t) times the steady f_x   (at x = chi(X_q, t))
__device__ __noinline__ void mms_source_unsteady(double X, double Y, double t, double amp, double rho, double mu,
                                                 double* fu, double* gp, double* fx) {
  const double pi = 3.14159265358979323846;
  const double st = sin(pi * t);
  const double s = sin(pi * X) * sin(pi * Y);
  const double x = X + amp * st * s, y = Y + amp * st * s;
  const double sx = sin(pi * x), cx = cos(pi * x), sy = sin(pi * y), cy = cos(pi * y);
  const double U1 = sx * cy, U2 = sx * sy;
  const double U1x = pi * cx * cy, U1y = -pi * sx * sy, U2x = pi * cx * sy, U2y = pi * sx * cy;
  const double lap1 = -2 * pi * pi * sx * cy, lap2 = -2 * pi * pi * sx * sy;
  const double gd1 = -pi * pi * sx * cy + pi * pi * cx * cy, gd2 = -pi * pi * cx * sy - pi * pi * sx * sy;
  const double Px = -pi * sx * cy, Py = -pi * cx * sy;
  const double t2 = t * t, t3 = t2 * t, t6 = t3 * t3;
  fu[0] = rho * (3 * t2 * U1 + t6 * (U1 * U1x + U2 * U1y)) + t2 * Px - mu * t3 * (lap1 + gd1);
  fu[1] = rho * (3 * t2 * U2 + t6 * (U1 * U2x + U2 * U2y)) + t2 * Py - mu * t3 * (lap2 + gd2);
  *gp = t3 * (U1x + U2y);
  const double f = amp * st * (4 * pi * pi * s - 2 * pi * pi * cos(pi * X) * cos(pi * Y));
  fx[0] = f;
  fx[1] = f;
}

// Coupled quasi-manufactured solution (Section 5.2) on the unit square around
// a rigid cylinder of radius R0 at X_c = (1/2, 1/2): with f = sin 2 pi t,
// d = amp (0.8, 0.6), x_c = X_c + f d, r = |x - x_c|, e = (x - x_c)/r and the
// kernel psi(r) = 1 - phi((r - R0)/(R1 - R0)), phi(s) = 6 s^5 - 15 s^4 + 10 s^3:
//   u = f' psi d,   p = A f psi (e.d) with A = -k/(pi R0),   x = X + f psi(|X - X_c|) d.
// Derivatives (e.d written ed, psi' and psi'' by r):
//   d_t u|_x      = f'' psi d - f'^2 psi' ed d          ((dr/dt = -f' ed)
//   (u.grad) u    = f'^2 psi psi' ed d
//   div u         = f' psi' ed,     lap u = f' (psi'' + psi'/r) d
//   grad div u    = f' [psi'' ed e + psi' (d - ed e)/r]
//   grad p        = A f [psi' ed e + psi (d - ed e)/r]
//   f_u = rho (d_t u + (u.grad) u) + grad p - mu (lap u + grad div u),  g_p = div u
//   f_x = -div_X sigma_s = -f [2 psi'' Ed E + 2 psi' (d - Ed E)/R + (psi'' + psi'/R) d]
//         (lambda_s = mu_s = 1; R = |X - X_c|, E = (X - X_c)/R, Ed = E.d)
constexpr double QUASI_CX = 0.5, QUASI_CY = 0.5, QUASI_R0 = 0.15, QUASI_R1 = 0.45;
constexpr double QUASI_DX = 0.8, QUASI_DY = 0.6;

__device__ __forceinline__ void quasi_kernel(double r, double& p0, double& p1, double& p2) {
  const double L = QUASI_R1 - QUASI_R0;
  const double s = fmin(1.0, fmax(0.0, (r - QUASI_R0) / L));
  p0 = 1.0 - s * s * s * (10.0 + s * (-15.0 + 6.0 * s));
  p1 = -30.0 * s * s * (s - 1.0) * (s - 1.0) / L;
  p2 = -60.0 * s * (s - 1.0) * (2.0 * s - 1.0) / (L * L);
}

__device__ __noinline__ void mms_source_quasi(double X, double Y, double t, double amp, double k, double rho,
                                              double mu, double* fu, double* gp, double* fx) {
  const double pi = 3.14159265358979323846;
  const double dx = amp * QUASI_DX, dy = amp * QUASI_DY;
  const double f = sin(2 * pi * t), f1 = 2 * pi * cos(2 * pi * t), f2 = -4 * pi * pi * f;
  // reference point: the mesh motion and the pseudo-solid source
  double Ex = X - QUASI_CX, Ey = Y - QUASI_CY;
  const double R = fmax(sqrt(Ex * Ex + Ey * Ey), 1e-12);
  Ex /= R;
  Ey /= R;
  double q0, q1, q2;
  quasi_kernel(R, q0, q1, q2);
  const double Ed = Ex * dx + Ey * dy;
  fx[0] = -f * (2 * q2 * Ed * Ex + 2 * q1 * (dx - Ed * Ex) / R + (q2 + q1 / R) * dx);
  fx[1] = -f * (2 * q2 * Ed * Ey + 2 * q1 * (dy - Ed * Ey) / R + (q2 + q1 / R) * dy);
  // physical point x = X + f psi(R) d and the fluid sources there
  const double x = X + f * q0 * dx, y = Y + f * q0 * dy;
  double ex = x - (QUASI_CX + f * dx), ey = y - (QUASI_CY + f * dy);
  const double r = fmax(sqrt(ex * ex + ey * ey), 1e-12);
  ex /= r;
  ey /= r;
  double p0, p1, p2;
  quasi_kernel(r, p0, p1, p2);
  const double ed = ex * dx + ey * dy;
  const double A = -k / (pi * QUASI_R0);
  const double dtu = f2 * p0, dtu_e = -f1 * f1 * p1 * ed;   // d_t u = (dtu + dtu_e) d
  const double conv = f1 * f1 * p0 * p1 * ed;               // (u.grad) u = conv d
  const double lap = f1 * (p2 + p1 / r);                   // lap u = lap d
  const double gd_e = f1 * p2 * ed, gd_d = f1 * p1 / r;     // grad div u = gd_e e + gd_d (d - ed e)
  const double gp_e = A * f * p1 * ed, gp_d = A * f * p0 / r;   // grad p = gp_e e + gp_d (d - ed e)
  const double tdx = dx - ed * ex, tdy = dy - ed * ey;
  fu[0] = rho * (dtu + dtu_e + conv) * dx + gp_e * ex + gp_d * tdx - mu * (lap * dx + gd_e * ex + gd_d * tdx);
  fu[1] = rho * (dtu + dtu_e + conv) * dy + gp_e * ey + gp_d * tdy - mu * (lap * dy + gd_e * ey + gd_d * tdy);
  *gp = f1 * p1 * ed;
}

template <class T>
__device__ void qp_compute(const Tables<T>& tb, const ElemNodes<T>& en, int q, T rho, T mu, int source,
                           double amp, double t_src, double k, T* out) {
  // current configuration
  T J00 = 0, J01 = 0, J10 = 0, J11 = 0;
  T K00 = 0, K01 = 0, K10 = 0, K11 = 0;   // reference
  for (int a = 0; a < 9; ++a) {
    T d0 = tb.dN[q][a][0], d1 = tb.dN[q][a][1];
    J00 += en.x[a][0] * d0; J01 += en.x[a][0] * d1;
    J10 += en.x[a][1] * d0; J11 += en.x[a][1] * d1;
    K00 += en.X[a][0] * d0; K01 += en.X[a][0] * d1;
    K10 += en.X[a][1] * d0; K11 += en.X[a][1] * d1;
  }
  T det = J00 * J11 - J01 * J10;
  T id = T(1) / det;
  T I00 = J11 * id, I01 = -J01 * id, I10 = -J10 * id, I11 = J00 * id;   // J^{-1}
  T det0 = K00 * K11 - K01 * K10;
  T id0 = T(1) / det0;
  T R00 = K11 * id0, R01 = -K01 * id0, R10 = -K10 * id0, R11 = K00 * id0;
  T u0 = 0, u1 = 0, w0 = 0, w1 = 0, ud0 = 0, ud1 = 0;
  T L00 = 0, L01 = 0, L10 = 0, L11 = 0;
  T F00 = 0, F01 = 0, F10 = 0, F11 = 0;   // grad_X of the displacement x - X
  for (int a = 0; a < 9; ++a) {
    T d0 = tb.dN[q][a][0], d1 = tb.dN[q][a][1];
    T g0 = d0 * I00 + d1 * I10, g1 = d0 * I01 + d1 * I11;   // g_a,i = sum_j dN_j Jinv_ji
    T r0 = d0 * R00 + d1 * R10, r1 = d0 * R01 + d1 * R11;
    out[Q_G + 2 * a] = g0;
    out[Q_G + 2 * a + 1] = g1;
    out[Q_G0 + 2 * a] = r0;
    out[Q_G0 + 2 * a + 1] = r1;
    T N = tb.N[q][a];
    u0 += N * en.u[a][0]; u1 += N * en.u[a][1];
    w0 += N * en.wn[a][0]; w1 += N * en.wn[a][1];
    ud0 += N * en.ud[a][0]; ud1 += N * en.ud[a][1];
    L00 += en.u[a][0] * g0; L01 += en.u[a][0] * g1;
    L10 += en.u[a][1] * g0; L11 += en.u[a][1] * g1;
    const T dx0 = en.x[a][0] - en.X[a][0], dx1 = en.x[a][1] - en.X[a][1];
    F00 += dx0 * r0; F01 += dx0 * r1;
    F10 += dx1 * r0; F11 += dx1 * r1;
  }
  T pq = 0;
  for (int c = 0; c < 4; ++c) pq += tb.M[q][c] * en.p[c];
  T uw0 = u0 - w0, uw1 = u1 - w1;
  out[Q_WDET] = tb.W[q] * det;
  out[Q_UW] = uw0;
  out[Q_UW + 1] = uw1;
  out[Q_L + 0] = L00; out[Q_L + 1] = L01; out[Q_L + 2] = L10; out[Q_L + 3] = L11;
  out[Q_SIG + 0] = -pq + 2 * mu * L00;
  out[Q_SIG + 1] = mu * (L01 + L10);
  out[Q_SIG + 2] = -pq + 2 * mu * L11;
  out[Q_INERT] = rho * (ud0 + uw0 * L00 + uw1 * L01);
  out[Q_INERT + 1] = rho * (ud1 + uw0 * L10 + uw1 * L11);
  out[Q_DIV] = L00 + L11;
  out[Q_WDET0] = tb.W[q] * det0 * en.lame;
  // eps = sym(grad_X x) - I = sym grad_X (x - X) since grad_X X = I
  T e00 = F00, e11 = F11, e01 = T(0.5) * (F01 + F10);
  out[Q_EPS] = e00; out[Q_EPS + 1] = e01; out[Q_EPS + 2] = e11;
  out[Q_TR] = e00 + e11;
  out[Q_FU] = out[Q_FU + 1] = out[Q_GP] = out[Q_FX] = out[Q_FX + 1] = T(0);
  if (source >= 1) {
    double Xq = 0, Yq = 0;
    for (int a = 0; a < 9; ++a) {
      Xq += (double)tb.N[q][a] * (double)en.X[a][0];
      Yq += (double)tb.N[q][a] * (double)en.X[a][1];
    }
    double fu[2], gp, fx[2];
    if (source == 1)
      mms_source(Xq, Yq, amp, (double)rho, (double)mu, fu, &gp, fx);
    else if (source == 2)
      mms_source_unsteady(Xq, Yq, t_src, amp, (double)rho, (double)mu, fu, &gp, fx);
    else
      mms_source_quasi(Xq, Yq, t_src, amp, k, (double)rho, (double)mu, fu, &gp, fx);
    out[Q_FU] = (T)fu[0];
    out[Q_FU + 1] = (T)fu[1];
    out[Q_GP] = (T)gp;
    out[Q_FX] = tb.W[q] * det0 * (T)fx[0];   // integrated over the reference element
    out[Q_FX + 1] = tb.W[q] * det0 * (T)fx[1];
  }
}

template <class T>
__device__ void load_element(const int32_t* conn, const double* X, const double* x,
                             const double* u, const double* p, const double* hu, const double* hx,
                             const double* lame, double c0, int e, int t, ElemNodes<T>& en) {
  // t in [0, 14): cooperative load by 14 threads of the element
  if (t < 9) {
    int nd = conn[e * 9 + t];
    for (int i = 0; i < 2; ++i) {
      double xv = x[2 * nd + i], uv = u[2 * nd + i];
      en.X[t][i] = (T)X[2 * nd + i];
      en.x[t][i] = (T)xv;
      en.u[t][i] = (T)uv;
      en.ud[t][i] = (T)(c0 * uv + hu[2 * nd + i]);
      en.wn[t][i] = (T)(c0 * xv + hx[2 * nd + i]);
    }
  } else if (t < 13) {
    const int vl[4] = {0, 2, 6, 8};
    en.p[t - 9] = (T)p[conn[e * 9 + vl[t - 9]]];
  } else if (t == 13) {
    en.lame = (T)lame[e];
  }
}

struct AsmArgs {
  const int32_t* conn;
  const int32_t* elems;     // elements of this colour
  int n;                    // count
  const double *X, *x, *u, *p, *hu, *hx, *lame;
  const int32_t* node_dof;
  const int32_t* e2nz;
  double rho, mu, k;
  int source;        // 0 none, 1 steady, 2 time-dependent, 3 coupled quasi-manufactured solution
  double source_amp;
  // device: {time of the step being solved, BDF rate coefficient c0} - read by
  // the kernels, so that captured CUDA graphs stay valid when either changes
  const double* step;
};

// Threads are laid out by row kind so that a warp runs one kind of row:
// [0, 18 EPB) momentum rows, [18 EPB, 22 EPB) continuity rows, [22 EPB, 40 EPB)
// pseudo-solid rows (element le = offset / rows of the kind).  Node loads use
// threads [0, 14 EPB), quadrature-point data threads [0, 9 EPB).
template <class T, bool JAC>
__global__ void __launch_bounds__(ASM_THREADS, 2) element_kernel(AsmArgs A, double* R, T* vals) {
  __shared__ Tables<T> tb;
  __shared__ ElemNodes<T> en[EPB];
  __shared__ T qd[EPB][9][QP_DATA];
  build_tables(tb);
  const int tid = threadIdx.x;
  if (tid < 14 * EPB) {
    const int le = tid / 14, gi = blockIdx.x * EPB + le;
    if (gi < A.n)
      load_element<T>(A.conn, A.X, A.x, A.u, A.p, A.hu, A.hx, A.lame, A.step[1], A.elems[gi], tid % 14, en[le]);
  }
  __syncthreads();
  if (tid < 9 * EPB) {
    const int le = tid / 9, q = tid % 9;
    if (blockIdx.x * EPB + le < A.n)
      qp_compute<T>(tb, en[le], q, (T)A.rho, (T)A.mu, A.source, A.source_amp, A.source >= 2 ? A.step[0] : 0.0,
                    A.k, qd[le][q]);
  }
  __syncthreads();
  int le, t;
  if (tid < 18 * EPB) {
    le = tid / 18;
    t = tid % 18;
  } else if (tid < 22 * EPB) {
    le = (tid - 18 * EPB) / 4;
    t = 18 + (tid - 18 * EPB) % 4;
  } else {
    le = (tid - 22 * EPB) / 18;
    t = 22 + (tid - 22 * EPB) % 18;
  }
  const int gi = blockIdx.x * EPB + le;
  if (gi >= A.n) return;
  const int e = A.elems[gi];
  const int* cn = A.conn + e * 9;
  const T c0 = (T)A.step[1], rho = (T)A.rho, mu = (T)A.mu;
  if (t < 18) {  // momentum row (a, i)
    const int a = t >> 1, i = t & 1;
    const int row = A.node_dof[cn[a] * NSLOT + i];
    if (row < 0) return;
    if (!JAC) {
      T acc = 0;
      for (int q = 0; q < 9; ++q) {
        const T* Q = qd[le][q];
        T ga0 = Q[Q_G + 2 * a], ga1 = Q[Q_G + 2 * a + 1];
        T s0 = i == 0 ? Q[Q_SIG + 0] : Q[Q_SIG + 1];
        T s1 = i == 0 ? Q[Q_SIG + 1] : Q[Q_SIG + 2];
        acc += Q[Q_WDET] * (tb.N[q][a] * (Q[Q_INERT + i] - Q[Q_FU + i]) + ga0 * s0 + ga1 * s1);
      }
      R[row] += (double)acc;
      return;
    }
    const int32_t* nz = A.e2nz + (int64_t)e * VOL_PAIRS;
    // u columns and x columns of node b
    for (int b = 0; b < 9; ++b) {
      T auu[2] = {0, 0}, aux[2] = {0, 0};
      for (int q = 0; q < 9; ++q) {
        const T* Q = qd[le][q];
        const T Na = tb.N[q][a], Nb = tb.N[q][b];
        const T ga0 = Q[Q_G + 2 * a], ga1 = Q[Q_G + 2 * a + 1];
        const T gb0 = Q[Q_G + 2 * b], gb1 = Q[Q_G + 2 * b + 1];
        const T wd = Q[Q_WDET];
        const T Li0 = Q[Q_L + 2 * i], Li1 = Q[Q_L + 2 * i + 1];          // L_i0, L_i1
        const T uwg = Q[Q_UW] * gb0 + Q[Q_UW + 1] * gb1;
        const T gagb = ga0 * gb0 + ga1 * gb1;
        const T gbi = i == 0 ? gb0 : gb1;
        const T si0 = i == 0 ? Q[Q_SIG + 0] : Q[Q_SIG + 1];
        const T si1 = i == 0 ? Q[Q_SIG + 1] : Q[Q_SIG + 2];
        const T sig_gb = si0 * gb0 + si1 * gb1;
        const T rai = Na * (Q[Q_INERT + i] - Q[Q_FU + i]) + ga0 * si0 + ga1 * si1;
        const T base = rho * Na * (c0 * Nb + uwg);
        for (int k = 0; k < 2; ++k) {
          const T Lik = k == 0 ? Li0 : Li1;
          const T gak = k == 0 ? ga0 : ga1;
          const T gbk = k == 0 ? gb0 : gb1;
          const T gaLk = ga0 * Q[Q_L + k] + ga1 * Q[Q_L + 2 + k];          // sum_j g_a,j L_jk
          T vu = rho * Na * Nb * Lik + mu * gak * gbi;
          if (k == i) vu += base + mu * gagb;
          auu[k] += wd * vu;
          T vx = -rho * Na * Lik * (c0 * Nb + uwg) - gak * sig_gb - mu * (Lik * gagb + gbi * gaLk) + rai * gbk;
          aux[k] += wd * vx;
        }
      }
      for (int k = 0; k < 2; ++k) {
        int s1 = nz[pairA(a, i, 4 * b + k)];
        if (s1 >= 0) vals[s1] += auu[k];
        int s2 = nz[pairA(a, i, 4 * b + 2 + k)];
        if (s2 >= 0) vals[s2] += aux[k];
      }
    }
    for (int c = 0; c < 4; ++c) {
      T acc = 0;
      for (int q = 0; q < 9; ++q) {
        const T* Q = qd[le][q];
        acc -= Q[Q_WDET] * Q[Q_G + 2 * a + i] * tb.M[q][c];
      }
      int s = nz[pairA(a, i, 36 + c)];
      if (s >= 0) vals[s] += acc;
    }
  } else if (t < 22) {  // continuity row c
    const int c = t - 18;
    const int vl[4] = {0, 2, 6, 8};
    const int row = A.node_dof[cn[vl[c]] * NSLOT + S_P];
    if (row < 0) return;
    if (!JAC) {
      T acc = 0;
      for (int q = 0; q < 9; ++q) acc -= qd[le][q][Q_WDET] * tb.M[q][c] * (qd[le][q][Q_DIV] - qd[le][q][Q_GP]);
      R[row] += (double)acc;
      return;
    }
    const int32_t* nz = A.e2nz + (int64_t)e * VOL_PAIRS;
    for (int b = 0; b < 9; ++b) {
      T au[2] = {0, 0}, ax[2] = {0, 0};
      for (int q = 0; q < 9; ++q) {
        const T* Q = qd[le][q];
        const T wm = Q[Q_WDET] * tb.M[q][c];
        const T gb0 = Q[Q_G + 2 * b], gb1 = Q[Q_G + 2 * b + 1];
        for (int k = 0; k < 2; ++k) {
          const T gbk = k == 0 ? gb0 : gb1;
          au[k] -= wm * gbk;
          const T Lg = Q[Q_L + k] * gb0 + Q[Q_L + 2 + k] * gb1;   // sum_i L_ik g_b,i
          ax[k] += wm * (Lg - (Q[Q_DIV] - Q[Q_GP]) * gbk);
        }
      }
      for (int k = 0; k < 2; ++k) {
        int s1 = nz[pairB(c, 4 * b + k)];
        if (s1 >= 0) vals[s1] += au[k];
        int s2 = nz[pairB(c, 4 * b + 2 + k)];
        if (s2 >= 0) vals[s2] += ax[k];
      }
    }
  } else {  // pseudo-solid row (a, i)
    const int r = t - 22;
    const int a = r >> 1, i = r & 1;
    const int row = A.node_dof[cn[a] * NSLOT + S_XX + i];
    if (row < 0) return;
    if (!JAC) {
      T acc = 0;
      for (int q = 0; q < 9; ++q) {
        const T* Q = qd[le][q];
        T ga0 = Q[Q_G0 + 2 * a], ga1 = Q[Q_G0 + 2 * a + 1];
        T gai = i == 0 ? ga0 : ga1;
        T e0 = i == 0 ? Q[Q_EPS] : Q[Q_EPS + 1];
        T e1 = i == 0 ? Q[Q_EPS + 1] : Q[Q_EPS + 2];
        acc += Q[Q_WDET0] * (gai * Q[Q_TR] + 2 * (ga0 * e0 + ga1 * e1)) - tb.N[q][a] * Q[Q_FX + i];
      }
      R[row] += (double)acc;
      return;
    }
    const int32_t* nz = A.e2nz + (int64_t)e * VOL_PAIRS;
    for (int b = 0; b < 9; ++b) {
      T ax[2] = {0, 0};
      for (int q = 0; q < 9; ++q) {
        const T* Q = qd[le][q];
        const T ga0 = Q[Q_G0 + 2 * a], ga1 = Q[Q_G0 + 2 * a + 1];
        const T gb0 = Q[Q_G0 + 2 * b], gb1 = Q[Q_G0 + 2 * b + 1];
        const T gai = i == 0 ? ga0 : ga1, gbi = i == 0 ? gb0 : gb1;
        const T gagb = ga0 * gb0 + ga1 * gb1;
        for (int k = 0; k < 2; ++k) {
          const T gak = k == 0 ? ga0 : ga1, gbk = k == 0 ? gb0 : gb1;
          T v = gai * gbk + gak * gbi;
          if (k == i) v += gagb;
          ax[k] += Q[Q_WDET0] * v;
        }
      }
      for (int k = 0; k < 2; ++k) {
        int s = nz[pairC(a, i, b, k)];
        if (s >= 0) vals[s] += ax[k];
      }
    }
  }
}

// ---- Gamma edges ----------------------------------------------------------------
struct FaceArgs {
  const int32_t* faces;     // F x 3 nodes
  const int32_t* list;      // faces of this colour
  int n;
  const double *x, *u, *lam, *hx;
  const int32_t* node_dof;
  const int32_t* f2nz;
  const double* step;   // device {time, c0} (see AsmArgs)
};

template <class T, bool JAC>
__global__ void face_kernel(FaceArgs A, double* R, T* vals) {
  int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= A.n) return;
  const double c0 = A.step[1];
  int f = A.list[gi];
  const int* fn = A.faces + 3 * f;
  double ds[3], N[3][3];
  double xb[3][2], ub[3][2], lb[3][2], wb[3][2];
  for (int b = 0; b < 3; ++b)
    for (int i = 0; i < 2; ++i) {
      xb[b][i] = A.x[2 * fn[b] + i];
      ub[b][i] = A.u[2 * fn[b] + i];
      lb[b][i] = A.lam[2 * fn[b] + i];
      wb[b][i] = c0 * xb[b][i] + A.hx[2 * fn[b] + i];
    }
  for (int q = 0; q < 3; ++q) {
    double L[3], dL[3];
    lag2(c_gpt[q], L, dL);
    double t0 = 0, t1 = 0;
    for (int b = 0; b < 3; ++b) {
      N[q][b] = L[b];
      t0 += dL[b] * xb[b][0];
      t1 += dL[b] * xb[b][1];
    }
    ds[q] = sqrt(t0 * t0 + t1 * t1) * c_gwt[q];
  }
  if (!JAC) {
    for (int b = 0; b < 3; ++b)
      for (int i = 0; i < 2; ++i) {
        double ru = 0, rl = 0;
        for (int q = 0; q < 3; ++q) {
          double lq = 0, uq = 0, wq = 0;
          for (int bp = 0; bp < 3; ++bp) {
            lq += N[q][bp] * lb[bp][i];
            uq += N[q][bp] * ub[bp][i];
            wq += N[q][bp] * wb[bp][i];
          }
          ru -= N[q][b] * lq * ds[q];
          rl -= N[q][b] * (uq - wq) * ds[q];
        }
        int du = A.node_dof[fn[b] * NSLOT + S_UX + i];
        if (du >= 0) R[du] += ru;
        int dl = A.node_dof[fn[b] * NSLOT + S_LX + i];
        if (dl >= 0) R[dl] += rl;
      }
    return;
  }
  const int32_t* nz = A.f2nz + (int64_t)f * FACE_PAIRS;
  for (int b = 0; b < 3; ++b)
    for (int bp = 0; bp < 3; ++bp) {
      double mass = 0, lin = 0;
      for (int q = 0; q < 3; ++q) mass += N[q][b] * N[q][bp] * ds[q];
      for (int q = 0; q < 3; ++q) lin += N[q][bp] * ds[q];
      for (int i = 0; i < 2; ++i) {
        int s;
        s = nz[fpairD(b, i, bp, i)];                   // d R[u_b,i] / d lambda_bp,i
        if (s >= 0) vals[s] += (T)(-mass);
        s = nz[fpairE(b, i, 2 * bp + i)];              // d R[lambda_b,i] / d u_bp,i
        if (s >= 0) vals[s] += (T)(-mass);
        s = nz[fpairE(b, i, 6 + 2 * bp + i)];          // d R[lambda_b,i] / d delta_i (w part)
        if (s >= 0) vals[s] += (T)(c0 * mass);
      }
      if (b == 0)
        for (int i = 0; i < 2; ++i) {
          int s = nz[fpairF(i, bp, i)];                // d R[delta_i] / d lambda_bp,i
          if (s >= 0) vals[s] += (T)lin;
        }
    }
}

// border rows: R[delta_i] = k delta_i + sum over Gamma of int lambda_i ds, in a
// fixed reduction order; with JAC the (delta_i, delta_i) entries get k
template <class T>
__global__ void border_kernel(const int32_t* faces, int nf, const double* x, const double* lam,
                              const double* delta, const int32_t* delta_dof, double k, double* R,
                              T* vals, int32_t dd0, int32_t dd1, bool jac) {
  __shared__ double red[2][256];
  double s0 = 0, s1 = 0;
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    const int* fn = faces + 3 * f;
    for (int q = 0; q < 3; ++q) {
      double L[3], dL[3];
      lag2(c_gpt[q], L, dL);
      double t0 = 0, t1 = 0, l0 = 0, l1 = 0;
      for (int b = 0; b < 3; ++b) {
        t0 += dL[b] * x[2 * fn[b]];
        t1 += dL[b] * x[2 * fn[b] + 1];
        l0 += L[b] * lam[2 * fn[b]];
        l1 += L[b] * lam[2 * fn[b] + 1];
      }
      double ds = sqrt(t0 * t0 + t1 * t1) * c_gwt[q];
      s0 += l0 * ds;
      s1 += l1 * ds;
    }
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && delta_dof[0] >= 0) {
    if (R) {
      R[delta_dof[0]] = k * delta[0] + red[0][0];
      R[delta_dof[1]] = k * delta[1] + red[1][0];
    }
    if (jac) {
      vals[dd0] += (T)k;
      vals[dd1] += (T)k;
    }
  }
}

__global__ void area_kernel(const int32_t* conn, const double* X, int64_t E, double scale, double* lame) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  double area = 0;
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) {
      double Li[3], dLi[3], Lj[3], dLj[3];
      lag2(c_gpt[i], Li, dLi);
      lag2(c_gpt[j], Lj, dLj);
      double J00 = 0, J01 = 0, J10 = 0, J11 = 0;
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          int nd = conn[e * 9 + 3 * b + a];
          double d0 = dLi[a] * Lj[b], d1 = Li[a] * dLj[b];
          J00 += X[2 * nd] * d0; J01 += X[2 * nd] * d1;
          J10 += X[2 * nd + 1] * d0; J11 += X[2 * nd + 1] * d1;
        }
      area += c_gwt[i] * c_gwt[j] * (J00 * J11 - J01 * J10);
    }
  lame[e] = area;
}

__global__ void min_kernel(const double* a, int64_t n, double* out) {
  __shared__ double red[256];
  double v = 1e300;
  for (int64_t i = threadIdx.x; i < n; i += 256) v = fmin(v, a[i]);
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// lambda_s = mu_s = scale * min|K_0| / |K_0|
__global__ void lame_kernel(double* lame, int64_t E, const double* amin, double scale) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < E) lame[e] = scale * (*amin) / lame[e];
}

}  // namespace

__global__ void fill_kernel(double* v, int64_t n, double a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] = a;
}

void launch_element_areas(const Mesh& m, double* lame, double scale, bool constant, double* scratch,
                          cudaStream_t s) {
  int E = (int)m.n_elems;
  if (constant) {   // lambda_s = mu_s = scale on every element
    Launched L(K_VEC, s);
    fill_kernel<<<(E + 255) / 256, 256, 0, s>>>(lame, E, scale);
    VIV_CUDA(cudaGetLastError());
    return;
  }
  if (m.dim == 3) {
    launch_element_volumes(m, lame, s);
  } else if (m.tri) {
    launch_triangle_areas(m, lame, s);
  } else {
    Launched L(K_VEC, s);
    area_kernel<<<(E + 127) / 128, 128, 0, s>>>(m.d_conn, m.d_X, E, scale, lame);
  }
  {
    Launched L(K_VEC, s);
    min_kernel<<<1, 256, 0, s>>>(lame, E, scratch);
  }
  {
    Launched L(K_VEC, s);
    lame_kernel<<<(E + 127) / 128, 128, 0, s>>>(lame, E, scratch, scale);
  }
  VIV_CUDA(cudaGetLastError());
}

// parts: 1 volume elements, 2 Gamma faces and border rows, 3 both
template <class T, bool JAC>
static void run_assembly(const Mesh& m, const CaseState& st, const vivParams& prm, double* R,
                         T* vals, cudaStream_t s, int parts = 3) {
  AsmArgs A;
  A.conn = m.d_conn;
  A.X = m.d_X;
  A.x = st.x;
  A.u = st.u;
  A.p = st.p;
  A.hu = st.hu;
  A.hx = st.hx;
  A.lame = st.lame;
  A.node_dof = m.d_node_dof;
  A.e2nz = m.d_e2nz;
  A.rho = prm.rho;
  A.mu = prm.mu;
  A.k = prm.k;
  A.source = prm.source;
  A.source_amp = prm.source_amp;
  A.step = st.step;
  if ((parts & 1) && m.tri) run_assembly_tri<T, JAC>(m, st, prm, R, vals, s);
  int ncol = (parts & 1) && !m.tri ? (int)m.color_off.size() - 1 : 0;
  for (int c = 0; c < ncol; ++c) {
    A.elems = m.d_color_elems + m.color_off[c];
    A.n = m.color_off[c + 1] - m.color_off[c];
    if (!A.n) continue;
    Launched L(JAC ? K_JAC : K_RES, s);
    element_kernel<T, JAC><<<(A.n + EPB - 1) / EPB, ASM_THREADS, 0, s>>>(A, R, vals);
  }
  FaceArgs Fa;
  Fa.faces = m.d_faces;
  Fa.x = st.x;
  Fa.u = st.u;
  Fa.lam = st.lam;
  Fa.hx = st.hx;
  Fa.node_dof = m.d_node_dof;
  Fa.f2nz = m.d_f2nz;
  Fa.step = st.step;
  if (!(parts & 2)) {
    VIV_CUDA(cudaGetLastError());
    return;
  }
  int nfc = (int)m.fcolor_off.size() - 1;
  for (int c = 0; c < nfc; ++c) {
    Fa.list = m.d_fcolor_faces + m.fcolor_off[c];
    Fa.n = m.fcolor_off[c + 1] - m.fcolor_off[c];
    if (!Fa.n) continue;
    Launched L(K_FACE, s);
    face_kernel<T, JAC><<<(Fa.n + 63) / 64, 64, 0, s>>>(Fa, R, vals);
  }
  if (m.n_faces > 0) {
    Launched L(K_FACE, s);
    border_kernel<T><<<1, 256, 0, s>>>(m.d_faces, (int)m.n_faces, st.x, st.lam, st.delta, m.d_delta_dof,
                                       prm.k, JAC ? nullptr : R, vals, m.dd_nz[0], m.dd_nz[1], JAC);
  }
  VIV_CUDA(cudaGetLastError());
}

void launch_residual(const Mesh& m, const CaseState& st, const vivParams& prm, cudaStream_t s) {
  VIV_CUDA(cudaMemsetAsync(st.R, 0, sizeof(double) * m.n_dofs, s));
  if (m.dim == 3)
    run_assembly3<double, false>(m, st, prm, st.R, (double*)nullptr, s, 3);
  else
    run_assembly<double, false>(m, st, prm, st.R, (double*)nullptr, s);
}

template <class T>
void launch_jacobian(const Mesh& m, const CaseState& st, const vivParams& prm, T* vals, cudaStream_t s) {
  VIV_CUDA(cudaMemsetAsync(vals, 0, sizeof(T) * m.row_ptr[m.n_dofs], s));
  if (m.dim == 3)
    run_assembly3<T, true>(m, st, prm, nullptr, vals, s, 3);
  else
    run_assembly<T, true>(m, st, prm, nullptr, vals, s);
}
template void launch_jacobian<double>(const Mesh&, const CaseState&, const vivParams&, double*, cudaStream_t);

// Volume element Jacobians in FP32 arithmetic; the Gamma-face and border
// (multiplier and cylinder position) entries in FP64.  Both arrays end up
// holding the same values (J64 exact widenings of the FP32 volume entries).
void launch_jacobian_split(const Mesh& m, const CaseState& st, const vivParams& prm, float* J32, double* J64,
                           cudaStream_t s) {
  const int64_t nnz = m.row_ptr[m.n_dofs];
  VIV_CUDA(cudaMemsetAsync(J32, 0, sizeof(float) * nnz, s));
  if (m.dim == 3)
    run_assembly3<float, true>(m, st, prm, nullptr, J32, s, 1);
  else
    run_assembly<float, true>(m, st, prm, nullptr, J32, s, 1);
  launch_f32_to_f64(J64, J32, nnz, s);
  if (m.dim == 3)
    run_assembly3<double, true>(m, st, prm, nullptr, J64, s, 2);
  else
    run_assembly<double, true>(m, st, prm, nullptr, J64, s, 2);
  launch_f64_to_f32(J32, J64, nnz, s);
}
template void launch_jacobian<float>(const Mesh&, const CaseState&, const vivParams&, float*, cudaStream_t);

// Exact Dirichlet data of the time-dependent manufactured solution at the
// step's time: prescribed velocity, position and pressure components
__global__ void mms_dirichlet_kernel(int64_t n, const int32_t* tags, const double* X, const double* step, double amp,
                                     double* u, double* x, double* p) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n) return;
  const double pi = 3.14159265358979323846, t = step[0];
  const double Xa = X[2 * a], Ya = X[2 * a + 1];
  const double b = amp * sin(pi * t) * sin(pi * Xa) * sin(pi * Ya);
  const double xa = Xa + b, ya = Ya + b;
  const int32_t tg = tags[a];
  const double t3 = t * t * t;
  if (tg & VIV_TAG_U_FIX_X) u[2 * a] = t3 * sin(pi * xa) * cos(pi * ya);
  if (tg & VIV_TAG_U_FIX_Y) u[2 * a + 1] = t3 * sin(pi * xa) * sin(pi * ya);
  if (tg & VIV_TAG_X_FIX_X) x[2 * a] = xa;
  if (tg & VIV_TAG_X_FIX_Y) x[2 * a + 1] = ya;
  if (tg & VIV_TAG_P_FIX) p[a] = t * t * cos(pi * xa) * cos(pi * ya);
}

__global__ void set_pair_kernel(double* dst, double a, double b) {
  dst[0] = a;
  dst[1] = b;
}

// the step's time and BDF rate coefficient, read by the assembly kernels
void launch_step_constants(const CaseState& st, double t_new, double c0, cudaStream_t s) {
  Launched L(K_VEC, s);
  set_pair_kernel<<<1, 1, 0, s>>>(st.step, t_new, c0);
  VIV_CUDA(cudaGetLastError());
}

void launch_mms_dirichlet(const Mesh& m, const CaseState& st, const vivParams& prm, cudaStream_t s) {
  Launched L(K_VEC, s);
  mms_dirichlet_kernel<<<(unsigned)((m.n_nodes + 255) / 256), 256, 0, s>>>(m.n_nodes, m.d_tags, m.d_X, st.step,
                                                                           prm.source_amp, st.u, st.x, st.p);
  VIV_CUDA(cudaGetLastError());
}

// initial velocity of the coupled quasi-manufactured solution: u(X, 0) = 2 pi psi(|X - X_c|) d
__global__ void quasi_init_kernel(int64_t n, const double* X, double amp, double* u) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n) return;
  const double pi = 3.14159265358979323846;
  const double ex = X[2 * a] - QUASI_CX, ey = X[2 * a + 1] - QUASI_CY;
  double q0, q1, q2;
  quasi_kernel(sqrt(ex * ex + ey * ey), q0, q1, q2);
  u[2 * a] = 2 * pi * q0 * amp * QUASI_DX;
  u[2 * a + 1] = 2 * pi * q0 * amp * QUASI_DY;
}

void launch_quasi_init(const Mesh& m, const CaseState& st, const vivParams& prm, cudaStream_t s) {
  Launched L(K_VEC, s);
  quasi_init_kernel<<<(unsigned)((m.n_nodes + 255) / 256), 256, 0, s>>>(m.n_nodes, m.d_X, prm.source_amp, st.u);
  VIV_CUDA(cudaGetLastError());
}

}  // namespace viv
