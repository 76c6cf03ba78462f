// Element kernels of the 3-D system: 27-node hexahedra (Q2 velocity and
// position, Q1 pressure on the 8 vertices) and 9-node faces of Gamma.
//
// The integrals are those of the 2-D kernels with three components
// (Eq. weak_system; nodal rates u_dot = c0 u + hu, w = c0 x + hx):
//   R[u_a,i] = int_Ot N_a rho (u_dot + ((u-w).grad)u)_i + grad N_a . sigma_i
//   R[p_c]   = -int_Ot M_c div u
//   R[x_a,i] = int_O0 lame ((grad_X N_a)_i tr eps + 2 grad_X N_a . eps_i),
//              eps = sym grad_X (x - X)
// Gamma faces: R[u_b,i] -= int N_b lambda_i dA, R[lambda_b,i] = -int N_b (u-w)_i dA,
// border rows R[delta_i] = k delta_i + int_Gamma lambda_i dA (i = x, y).
// Periodic span: a node whose bit is set in the element's wrap mask sits at
// its stored coordinates + span e_z (reference and current); the mesh
// velocity is formed from the stored positions.
//
// Jacobian: the analytic derivative including the shape derivatives (the
// same identities as in 2-D, with k over three components): d(det J) =
// det J g_b,k, d(g_a,j) = -g_a,k g_b,j, d(L_ij) = -L_ik g_b,j, d(w) = c0 N_b e_k.
// On Gamma the x, y position columns are delta's and the z position is held;
// a rigid shift of a face leaves its area element unchanged, so the face rows
// have no position derivative other than the mesh velocity's.
//
// One CTA per element: the Gauss-point geometry is built in shared memory
// by (point, node) pairs, then one thread per element row computes all of
// its columns and scatters them through e2nz.  Elements of one colour share
// no node, so one colour per launch needs no atomics (deterministic sums).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "viv_internal.h"

namespace viv {
namespace {

constexpr int NP = 27;        // nodes per hexahedron
constexpr int NQ = 27;        // 3 x 3 x 3 Gauss points
constexpr int NV = 8;         // pressure vertices
constexpr int THREADS3 = 192; // 170 element rows: 81 momentum, 8 continuity, 81 pseudo-solid
constexpr int TAB_SIZE = NQ * NP + NQ * NP * 3 + NQ * NV + NQ;   // 3,159

template <class T>
struct Tab3 {
  T N[NQ][NP];
  T dN[NQ][NP][3];
  T M[NQ][NV];
  T W[NQ];
};
static_assert(sizeof(Tab3<double>) == TAB_SIZE * sizeof(double), "table layout");

template <class T>
struct Nodes3 {
  T X[NP][3], x[NP][3], u[NP][3], ud[NP][3], wn[NP][3], p[NV];
  T lame;
};

// per Gauss point record; symmetric tensors as 00 01 02 11 12 22
enum {
  R_WDET = 0, R_G = 1, R_UW = 82, R_L = 85, R_SIG = 94, R_INERT = 100, R_DIV = 103,
  R_WDET0 = 104, R_G0 = 105, R_EPS = 186, R_TR = 192, R_JI = 193, R_JI0 = 202, QREC = 211
};

__host__ __device__ __forceinline__ int sym3(int i, int j) {
  return i <= j ? (i == 0 ? j : (i == 1 ? 2 + j : 5)) : (j == 0 ? i : (j == 1 ? 2 + i : 5));
}

__host__ __device__ __forceinline__ int vertex_node(int c) { return 18 * (c >> 2) + 6 * ((c >> 1) & 1) + 2 * (c & 1); }

template <class T>
size_t hex_smem_bytes() {
  return sizeof(Tab3<T>) + sizeof(Nodes3<T>) + (size_t)NQ * QREC * sizeof(T);
}

struct Asm3Args {
  const int32_t* conn;
  const int32_t* wrap;
  const int32_t* elems;     // elements of this colour
  const void* tab;          // Tab3<T> in global memory
  double span;
  const double *X, *x, *u, *p, *hu, *hx, *lame;
  const int32_t* node_dof;
  const int32_t* e2nz;
  double rho, mu;
  const double* step;       // device {time, c0}
};

template <class T, bool JAC>
__global__ void __launch_bounds__(THREADS3) hex_kernel(Asm3Args A, double* R, T* vals) {
  extern __shared__ __align__(16) unsigned char smem[];
  Tab3<T>& tb = *reinterpret_cast<Tab3<T>*>(smem);
  Nodes3<T>& en = *reinterpret_cast<Nodes3<T>*>(smem + sizeof(Tab3<T>));
  T* qd = reinterpret_cast<T*>(smem + sizeof(Tab3<T>) + sizeof(Nodes3<T>));
  const int tid = threadIdx.x;
  {
    const T* gt = static_cast<const T*>(A.tab);
    T* st = reinterpret_cast<T*>(&tb);
    for (int i = tid; i < TAB_SIZE; i += THREADS3) st[i] = gt[i];
  }
  const int e = A.elems[blockIdx.x];
  const int32_t* cn = A.conn + (int64_t)e * NP;
  const double c0d = A.step[1];
  if (tid < NP) {
    const int nd = cn[tid];
    const double sz = (A.wrap[e] >> tid & 1) ? A.span : 0.0;
    for (int i = 0; i < 3; ++i) {
      const double xv = A.x[3 * nd + i], uv = A.u[3 * nd + i];
      const double sh = i == 2 ? sz : 0.0;
      en.X[tid][i] = (T)(A.X[3 * nd + i] + sh);
      en.x[tid][i] = (T)(xv + sh);
      en.u[tid][i] = (T)uv;
      en.ud[tid][i] = (T)(c0d * uv + A.hu[3 * nd + i]);
      en.wn[tid][i] = (T)(c0d * xv + A.hx[3 * nd + i]);
    }
  } else if (tid < NP + NV) {
    en.p[tid - NP] = (T)A.p[cn[vertex_node(tid - NP)]];
  } else if (tid == NP + NV) {
    en.lame = (T)A.lame[e];
  }
  __syncthreads();
  // (A) Jacobian matrices of the current and reference maps, inverses, weights
  if (tid < 2 * NQ) {
    const int q = tid % NQ;
    const bool ref = tid >= NQ;
    T J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < NP; ++a)
      for (int i = 0; i < 3; ++i) {
        const T c = ref ? en.X[a][i] : en.x[a][i];
        for (int j = 0; j < 3; ++j) J[i][j] += c * tb.dN[q][a][j];
      }
    const T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const T det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const T id = T(1) / det;
    T* Q = qd + q * QREC;
    T* Ji = Q + (ref ? R_JI0 : R_JI);   // Jinv[j][i] at 3 j + i
    Ji[0] = c00 * id;
    Ji[3] = c01 * id;
    Ji[6] = c02 * id;
    Ji[1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[4] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[7] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[5] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[8] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    if (ref)
      Q[R_WDET0] = tb.W[q] * det * en.lame;
    else
      Q[R_WDET] = tb.W[q] * det;
  }
  __syncthreads();
  // (B) physical gradients g_a = J^{-T} grad_xi N_a, current and reference
  for (int t = tid; t < NQ * NP; t += THREADS3) {
    const int q = t / NP, a = t % NP;
    T* Q = qd + q * QREC;
    const T d0 = tb.dN[q][a][0], d1 = tb.dN[q][a][1], d2 = tb.dN[q][a][2];
    for (int i = 0; i < 3; ++i) {
      Q[R_G + 3 * a + i] = d0 * Q[R_JI + i] + d1 * Q[R_JI + 3 + i] + d2 * Q[R_JI + 6 + i];
      Q[R_G0 + 3 * a + i] = d0 * Q[R_JI0 + i] + d1 * Q[R_JI0 + 3 + i] + d2 * Q[R_JI0 + 6 + i];
    }
  }
  __syncthreads();
  // (C) fields at the Gauss points
  if (tid < NQ) {
    const int q = tid;
    T* Q = qd + q * QREC;
    const T mu = (T)A.mu, rho = (T)A.rho;
    T u[3] = {0, 0, 0}, w[3] = {0, 0, 0}, ud[3] = {0, 0, 0};
    T L[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, F[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < NP; ++a) {
      const T N = tb.N[q][a];
      const T* g = Q + R_G + 3 * a;
      const T* g0 = Q + R_G0 + 3 * a;
      for (int i = 0; i < 3; ++i) {
        u[i] += N * en.u[a][i];
        w[i] += N * en.wn[a][i];
        ud[i] += N * en.ud[a][i];
        const T dxi = en.x[a][i] - en.X[a][i];
        for (int j = 0; j < 3; ++j) {
          L[i][j] += en.u[a][i] * g[j];
          F[i][j] += dxi * g0[j];
        }
      }
    }
    T pq = 0;
    for (int c = 0; c < NV; ++c) pq += tb.M[q][c] * en.p[c];
    T uw[3];
    for (int i = 0; i < 3; ++i) {
      uw[i] = u[i] - w[i];
      Q[R_UW + i] = uw[i];
      for (int j = 0; j < 3; ++j) Q[R_L + 3 * i + j] = L[i][j];
    }
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) {
        Q[R_SIG + sym3(i, j)] = mu * (L[i][j] + L[j][i]) - (i == j ? pq : T(0));
        Q[R_EPS + sym3(i, j)] = T(0.5) * (F[i][j] + F[j][i]);
      }
    for (int i = 0; i < 3; ++i) Q[R_INERT + i] = rho * (ud[i] + L[i][0] * uw[0] + L[i][1] * uw[1] + L[i][2] * uw[2]);
    Q[R_DIV] = L[0][0] + L[1][1] + L[2][2];
    Q[R_TR] = F[0][0] + F[1][1] + F[2][2];
  }
  __syncthreads();
  if (tid >= 170) return;
  const T c0 = (T)c0d, rho = (T)A.rho, mu = (T)A.mu;
  const int32_t* nz = A.e2nz + (int64_t)e * VOL_PAIRS3;
  if (tid < 81) {  // momentum row (a, i)
    const int a = tid / 3, i = tid % 3;
    const int row = A.node_dof[cn[a] * NSLOT + S_UX + i];
    if (row < 0) return;
    if (!JAC) {
      T acc = 0;
      for (int q = 0; q < NQ; ++q) {
        const T* Q = qd + q * QREC;
        const T* ga = Q + R_G + 3 * a;
        acc += Q[R_WDET] * (tb.N[q][a] * Q[R_INERT + i] + ga[0] * Q[R_SIG + sym3(i, 0)] +
                            ga[1] * Q[R_SIG + sym3(i, 1)] + ga[2] * Q[R_SIG + sym3(i, 2)]);
      }
      R[row] += (double)acc;
      return;
    }
    for (int b = 0; b < NP; ++b) {
      T auu[3] = {0, 0, 0}, aux[3] = {0, 0, 0};
      for (int q = 0; q < NQ; ++q) {
        const T* Q = qd + q * QREC;
        const T Na = tb.N[q][a], Nb = tb.N[q][b];
        const T ga[3] = {Q[R_G + 3 * a], Q[R_G + 3 * a + 1], Q[R_G + 3 * a + 2]};
        const T gb[3] = {Q[R_G + 3 * b], Q[R_G + 3 * b + 1], Q[R_G + 3 * b + 2]};
        const T wd = Q[R_WDET];
        const T Li[3] = {Q[R_L + 3 * i], Q[R_L + 3 * i + 1], Q[R_L + 3 * i + 2]};
        const T si[3] = {Q[R_SIG + sym3(i, 0)], Q[R_SIG + sym3(i, 1)], Q[R_SIG + sym3(i, 2)]};
        const T uwg = Q[R_UW] * gb[0] + Q[R_UW + 1] * gb[1] + Q[R_UW + 2] * gb[2];
        const T gagb = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
        const T gbi = gb[i];
        const T sig_gb = si[0] * gb[0] + si[1] * gb[1] + si[2] * gb[2];
        const T rai = Na * Q[R_INERT + i] + ga[0] * si[0] + ga[1] * si[1] + ga[2] * si[2];
        const T cnb = c0 * Nb + uwg;
        for (int k = 0; k < 3; ++k) {
          const T gaLk = ga[0] * Q[R_L + k] + ga[1] * Q[R_L + 3 + k] + ga[2] * Q[R_L + 6 + k];
          T vu = rho * Na * Nb * Li[k] + mu * ga[k] * gbi;
          if (k == i) vu += rho * Na * cnb + mu * gagb;
          auu[k] += wd * vu;
          const T vx = -rho * Na * Li[k] * cnb - ga[k] * sig_gb - mu * (Li[k] * gagb + gbi * gaLk) + rai * gb[k];
          aux[k] += wd * vx;
        }
      }
      for (int k = 0; k < 3; ++k) {
        const int s1 = nz[pairA3(a, i, 6 * b + k)];
        if (s1 >= 0) vals[s1] += auu[k];
        const int s2 = nz[pairA3(a, i, 6 * b + 3 + k)];
        if (s2 >= 0) vals[s2] += aux[k];
      }
    }
    for (int c = 0; c < NV; ++c) {
      T acc = 0;
      for (int q = 0; q < NQ; ++q) {
        const T* Q = qd + q * QREC;
        acc -= Q[R_WDET] * Q[R_G + 3 * a + i] * tb.M[q][c];
      }
      const int s = nz[pairA3(a, i, 162 + c)];
      if (s >= 0) vals[s] += acc;
    }
  } else if (tid < 89) {  // continuity row c
    const int c = tid - 81;
    const int row = A.node_dof[cn[vertex_node(c)] * NSLOT + S_P];
    if (row < 0) return;
    if (!JAC) {
      T acc = 0;
      for (int q = 0; q < NQ; ++q) acc -= qd[q * QREC + R_WDET] * tb.M[q][c] * qd[q * QREC + R_DIV];
      R[row] += (double)acc;
      return;
    }
    for (int b = 0; b < NP; ++b) {
      T au[3] = {0, 0, 0}, ax[3] = {0, 0, 0};
      for (int q = 0; q < NQ; ++q) {
        const T* Q = qd + q * QREC;
        const T wm = Q[R_WDET] * tb.M[q][c];
        const T gb[3] = {Q[R_G + 3 * b], Q[R_G + 3 * b + 1], Q[R_G + 3 * b + 2]};
        for (int k = 0; k < 3; ++k) {
          au[k] -= wm * gb[k];
          const T Lg = Q[R_L + k] * gb[0] + Q[R_L + 3 + k] * gb[1] + Q[R_L + 6 + k] * gb[2];   // sum_i L_ik g_b,i
          ax[k] += wm * (Lg - Q[R_DIV] * gb[k]);
        }
      }
      for (int k = 0; k < 3; ++k) {
        const int s1 = nz[pairB3(c, 6 * b + k)];
        if (s1 >= 0) vals[s1] += au[k];
        const int s2 = nz[pairB3(c, 6 * b + 3 + k)];
        if (s2 >= 0) vals[s2] += ax[k];
      }
    }
  } else {  // pseudo-solid row (a, i)
    const int r = tid - 89;
    const int a = r / 3, i = r % 3;
    const int row = A.node_dof[cn[a] * NSLOT + S_XX + i];
    if (row < 0) return;
    if (!JAC) {
      T acc = 0;
      for (int q = 0; q < NQ; ++q) {
        const T* Q = qd + q * QREC;
        const T* ga = Q + R_G0 + 3 * a;
        acc += Q[R_WDET0] * (ga[i] * Q[R_TR] + 2 * (ga[0] * Q[R_EPS + sym3(i, 0)] + ga[1] * Q[R_EPS + sym3(i, 1)] +
                                                     ga[2] * Q[R_EPS + sym3(i, 2)]));
      }
      R[row] += (double)acc;
      return;
    }
    for (int b = 0; b < NP; ++b) {
      T ax[3] = {0, 0, 0};
      for (int q = 0; q < NQ; ++q) {
        const T* Q = qd + q * QREC;
        const T ga[3] = {Q[R_G0 + 3 * a], Q[R_G0 + 3 * a + 1], Q[R_G0 + 3 * a + 2]};
        const T gb[3] = {Q[R_G0 + 3 * b], Q[R_G0 + 3 * b + 1], Q[R_G0 + 3 * b + 2]};
        const T gagb = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
        for (int k = 0; k < 3; ++k) {
          T v = ga[i] * gb[k] + ga[k] * gb[i];
          if (k == i) v += gagb;
          ax[k] += Q[R_WDET0] * v;
        }
      }
      for (int k = 0; k < 3; ++k) {
        const int s = nz[pairC3(a, i, b, k)];
        if (s >= 0) vals[s] += ax[k];
      }
    }
  }
}

__device__ __forceinline__ void lag2d(double s, double* L, double* dL) {
  L[0] = (1 - s) * (1 - 2 * s);
  L[1] = 4 * s * (1 - s);
  L[2] = s * (2 * s - 1);
  dL[0] = 4 * s - 3;
  dL[1] = 4 - 8 * s;
  dL[2] = 4 * s - 1;
}

__device__ __constant__ double g3pt[3] = {0.11270166537925831148, 0.5, 0.88729833462074168852};
__device__ __constant__ double g3wt[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};

// area element data of a 9-node face at its 3 x 3 Gauss points (FP64)
__device__ void face_geometry(const double (&xb)[9][3], double (&N)[9][9], double (&dA)[9]) {
  for (int qt = 0; qt < 3; ++qt)
    for (int qs = 0; qs < 3; ++qs) {
      const int q = 3 * qt + qs;
      double Ls[3], dLs[3], Lt[3], dLt[3];
      lag2d(g3pt[qs], Ls, dLs);
      lag2d(g3pt[qt], Lt, dLt);
      double t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
      for (int bt = 0; bt < 3; ++bt)
        for (int bs = 0; bs < 3; ++bs) {
          const int b = 3 * bt + bs;
          N[q][b] = Ls[bs] * Lt[bt];
          for (int i = 0; i < 3; ++i) {
            t1[i] += dLs[bs] * Lt[bt] * xb[b][i];
            t2[i] += Ls[bs] * dLt[bt] * xb[b][i];
          }
        }
      const double n0 = t1[1] * t2[2] - t1[2] * t2[1];
      const double n1 = t1[2] * t2[0] - t1[0] * t2[2];
      const double n2 = t1[0] * t2[1] - t1[1] * t2[0];
      dA[q] = sqrt(n0 * n0 + n1 * n1 + n2 * n2) * g3wt[qs] * g3wt[qt];
    }
}

struct Face3Args {
  const int32_t* faces;     // F x 9 nodes
  const int32_t* fwrap;     // per face, bit b: node b at X + span e_z
  const int32_t* list;      // faces of this colour
  int n;
  double span;
  const double *x, *u, *lam, *hx;
  const int32_t* node_dof;
  const int32_t* f2nz;
  const double* step;
};

template <class T, bool JAC>
__global__ void face3_kernel(Face3Args A, double* R, T* vals) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= A.n) return;
  const double c0 = A.step[1];
  const int f = A.list[gi];
  const int* fn = A.faces + 9 * f;
  double xb[9][3];
  for (int b = 0; b < 9; ++b) {
    for (int i = 0; i < 3; ++i) xb[b][i] = A.x[3 * fn[b] + i];
    if (A.fwrap[f] >> b & 1) xb[b][2] += A.span;
  }
  double N[9][9], dA[9];
  face_geometry(xb, N, dA);
  if (!JAC) {
    for (int b = 0; b < 9; ++b)
      for (int i = 0; i < 3; ++i) {
        double ru = 0, rl = 0;
        for (int q = 0; q < 9; ++q) {
          double lq = 0, uwq = 0;
          for (int bp = 0; bp < 9; ++bp) {
            const int nd = fn[bp];
            lq += N[q][bp] * A.lam[3 * nd + i];
            uwq += N[q][bp] * (A.u[3 * nd + i] - (c0 * A.x[3 * nd + i] + A.hx[3 * nd + i]));
          }
          ru -= N[q][b] * lq * dA[q];
          rl -= N[q][b] * uwq * dA[q];
        }
        const int du = A.node_dof[fn[b] * NSLOT + S_UX + i];
        if (du >= 0) R[du] += ru;
        const int dl = A.node_dof[fn[b] * NSLOT + S_LX + i];
        if (dl >= 0) R[dl] += rl;
      }
    return;
  }
  const int32_t* nz = A.f2nz + (int64_t)f * FACE_PAIRS3;
  for (int b = 0; b < 9; ++b) {
    double wsum = 0;
    for (int bp = 0; bp < 9; ++bp) {
      double mass = 0;
      for (int q = 0; q < 9; ++q) mass += N[q][b] * N[q][bp] * dA[q];
      wsum += mass;
      for (int i = 0; i < 3; ++i) {
        int s = nz[fpairD3(b, i, bp)];   // d R[u_b,i] / d lambda_bp,i
        if (s >= 0) vals[s] += (T)(-mass);
        s = nz[fpairE3(b, i, bp)];       // d R[lambda_b,i] / d u_bp,i
        if (s >= 0) vals[s] += (T)(-mass);
      }
    }
    for (int i = 0; i < 2; ++i) {        // d R[lambda_b,i] / d delta_i: the mesh velocity c0 x
      const int s = nz[fpairG3(b, i)];
      if (s >= 0) vals[s] += (T)(c0 * wsum);
    }
  }
  for (int bp = 0; bp < 9; ++bp) {
    double lin = 0;
    for (int q = 0; q < 9; ++q) lin += N[q][bp] * dA[q];
    for (int i = 0; i < 2; ++i) {        // d R[delta_i] / d lambda_bp,i
      const int s = nz[fpairF3(i, bp)];
      if (s >= 0) vals[s] += (T)lin;
    }
  }
}

// border rows: R[delta_i] = k delta_i + sum over Gamma of int lambda_i dA in a
// fixed reduction order; with JAC the (delta_i, delta_i) entries get k
template <class T>
__global__ void border3_kernel(const int32_t* faces, const int32_t* fwrap, int nf, double span, const double* x,
                               const double* lam, const double* delta, const int32_t* delta_dof, double k,
                               double* R, T* vals, int32_t dd0, int32_t dd1, bool jac) {
  __shared__ double red[2][256];
  double s0 = 0, s1 = 0;
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    const int* fn = faces + 9 * f;
    double xb[9][3];
    for (int b = 0; b < 9; ++b) {
      for (int i = 0; i < 3; ++i) xb[b][i] = x[3 * fn[b] + i];
      if (fwrap[f] >> b & 1) xb[b][2] += span;
    }
    double N[9][9], dA[9];
    face_geometry(xb, N, dA);
    for (int q = 0; q < 9; ++q) {
      double l0 = 0, l1 = 0;
      for (int b = 0; b < 9; ++b) {
        l0 += N[q][b] * lam[3 * fn[b]];
        l1 += N[q][b] * lam[3 * fn[b] + 1];
      }
      s0 += l0 * dA[q];
      s1 += l1 * dA[q];
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

// reference volume |K_0| of each hexahedron (seam-shifted coordinates)
__global__ void volume3_kernel(const int32_t* conn, const int32_t* wrap, double span, const double* X, int64_t E,
                               double* vol) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  double v = 0;
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) {
        double Li[3], dLi[3], Lj[3], dLj[3], Lk[3], dLk[3];
        lag2d(g3pt[i], Li, dLi);
        lag2d(g3pt[j], Lj, dLj);
        lag2d(g3pt[k], Lk, dLk);
        double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int c = 0; c < 3; ++c)
          for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
              const int loc = 9 * c + 3 * b + a;
              const int nd = conn[e * 27 + loc];
              const double d[3] = {dLi[a] * Lj[b] * Lk[c], Li[a] * dLj[b] * Lk[c], Li[a] * Lj[b] * dLk[c]};
              for (int r = 0; r < 3; ++r) {
                const double xr = X[3 * nd + r] + ((r == 2 && (wrap[e] >> loc & 1)) ? span : 0.0);
                for (int s = 0; s < 3; ++s) J[r][s] += xr * d[s];
              }
            }
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        v += g3wt[i] * g3wt[j] * g3wt[k] * det;
      }
  vol[e] = v;
}

// shape-function tables at the Gauss points (host, FP64), layout of Tab3
std::vector<double> hex_tables_host() {
  const double g = std::sqrt(15.0) / 10.0;
  const double pts[3] = {0.5 - g, 0.5, 0.5 + g};
  const double wts[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  auto lag = [](double s, double* L, double* dL) {
    L[0] = (1 - s) * (1 - 2 * s);
    L[1] = 4 * s * (1 - s);
    L[2] = s * (2 * s - 1);
    dL[0] = 4 * s - 3;
    dL[1] = 4 - 8 * s;
    dL[2] = 4 * s - 1;
  };
  Tab3<double> t;
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) {
        const int q = 9 * k + 3 * j + i;
        double Li[3], dLi[3], Lj[3], dLj[3], Lk[3], dLk[3];
        lag(pts[i], Li, dLi);
        lag(pts[j], Lj, dLj);
        lag(pts[k], Lk, dLk);
        t.W[q] = wts[i] * wts[j] * wts[k];
        for (int c = 0; c < 3; ++c)
          for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
              const int n = 9 * c + 3 * b + a;
              t.N[q][n] = Li[a] * Lj[b] * Lk[c];
              t.dN[q][n][0] = dLi[a] * Lj[b] * Lk[c];
              t.dN[q][n][1] = Li[a] * dLj[b] * Lk[c];
              t.dN[q][n][2] = Li[a] * Lj[b] * dLk[c];
            }
        const double l1[2][3] = {{1 - pts[i], 1 - pts[j], 1 - pts[k]}, {pts[i], pts[j], pts[k]}};
        for (int cv = 0; cv < NV; ++cv) t.M[q][cv] = l1[cv & 1][0] * l1[(cv >> 1) & 1][1] * l1[cv >> 2][2];
      }
  const double* p = reinterpret_cast<const double*>(&t);
  return std::vector<double>(p, p + TAB_SIZE);
}

template <class T, bool JAC>
void set_hex_smem() {
  VIV_CUDA(cudaFuncSetAttribute(hex_kernel<T, JAC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)hex_smem_bytes<T>()));
}

}  // namespace

// the element kernels' shared-memory limit, once per device before any launch
// (case creation; the serving loop's worker threads may get here concurrently)
void prepare_hex_kernels() {
  constexpr int MAX_DEV = 64;
  static std::once_flag once[MAX_DEV];
  int dev = 0;
  VIV_CUDA(cudaGetDevice(&dev));
  VIV_CHECK(dev >= 0 && dev < MAX_DEV, VIV_ERR_ARG, "device index out of range");
  std::call_once(once[dev], [] {
    set_hex_smem<double, false>();
    set_hex_smem<double, true>();
    set_hex_smem<float, true>();
  });
}

void upload_hex_tables(Mesh& m, cudaStream_t s) {
  std::vector<double> t = hex_tables_host();
  std::vector<float> tf(t.begin(), t.end());
  m.d_hex_tab = m.arena.upload(t, s);
  m.d_hex_tab_f = m.arena.upload(tf, s);
}

void launch_element_volumes(const Mesh& m, double* vol, cudaStream_t s) {
  Launched L(K_VEC, s);
  volume3_kernel<<<(unsigned)((m.n_elems + 127) / 128), 128, 0, s>>>(m.d_conn, m.d_wrap, m.span, m.d_X, m.n_elems,
                                                                     vol);
  VIV_CUDA(cudaGetLastError());
}

// parts: 1 volume elements, 2 Gamma faces and border rows, 3 both
template <class T, bool JAC>
void run_assembly3(const Mesh& m, const CaseState& st, const vivParams& prm, double* R, T* vals, cudaStream_t s,
                   int parts) {
  if (parts & 1) {
    prepare_hex_kernels();
    Asm3Args A;
    A.conn = m.d_conn;
    A.wrap = m.d_wrap;
    A.tab = std::is_same<T, float>::value ? (const void*)m.d_hex_tab_f : (const void*)m.d_hex_tab;
    A.span = m.span;
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
    A.step = st.step;
    const size_t smem = hex_smem_bytes<T>();
    for (int c = 0; c + 1 < (int)m.color_off.size(); ++c) {
      const int n = m.color_off[c + 1] - m.color_off[c];
      if (!n) continue;
      A.elems = m.d_color_elems + m.color_off[c];
      Launched L(JAC ? K_JAC : K_RES, s);
      hex_kernel<T, JAC><<<n, THREADS3, smem, s>>>(A, R, vals);
    }
  }
  if ((parts & 2) && m.n_faces > 0) {
    Face3Args F;
    F.faces = m.d_faces;
    F.fwrap = m.d_face_wrap;
    F.span = m.span;
    F.x = st.x;
    F.u = st.u;
    F.lam = st.lam;
    F.hx = st.hx;
    F.node_dof = m.d_node_dof;
    F.f2nz = m.d_f2nz;
    F.step = st.step;
    for (int c = 0; c + 1 < (int)m.fcolor_off.size(); ++c) {
      F.list = m.d_fcolor_faces + m.fcolor_off[c];
      F.n = m.fcolor_off[c + 1] - m.fcolor_off[c];
      if (!F.n) continue;
      Launched L(K_FACE, s);
      face3_kernel<T, JAC><<<(F.n + 63) / 64, 64, 0, s>>>(F, R, vals);
    }
    Launched L(K_FACE, s);
    border3_kernel<T><<<1, 256, 0, s>>>(m.d_faces, m.d_face_wrap, (int)m.n_faces, m.span, st.x, st.lam, st.delta,
                                        m.d_delta_dof, prm.k, JAC ? nullptr : R, vals, m.dd_nz[0], m.dd_nz[1], JAC);
  }
  VIV_CUDA(cudaGetLastError());
}

template void run_assembly3<double, false>(const Mesh&, const CaseState&, const vivParams&, double*, double*,
                                           cudaStream_t, int);
template void run_assembly3<double, true>(const Mesh&, const CaseState&, const vivParams&, double*, double*,
                                          cudaStream_t, int);
template void run_assembly3<float, true>(const Mesh&, const CaseState&, const vivParams&, double*, float*,
                                         cudaStream_t, int);

}  // namespace viv
