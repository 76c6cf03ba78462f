// Element kernels of the paper's own discretisation (Section 3.3): Taylor-Hood
// P2-P1 triangles (6-node velocity, pressure on the vertices) with a P1 mesh
// position (position unknowns on the vertices; straight edges, an affine map
// per triangle).
//
// The integrals are those of the Q2 kernels (Eq. weak_system), with the mesh
// velocity the P1 interpolant of the vertex rates w_v = c0 x_v + hx_v:
//   R[u_a,i] = int_Ot N_a rho (u_dot + ((u-w).grad)u)_i + grad N_a . sigma_i
//   R[p_c]   = -int_Ot M_c div u
//   R[x_v,i] = int_O0 lame ((grad_X M_v)_i tr eps + 2 grad_X M_v . eps_i)
// (eps = sym grad_X (x - X) is constant per triangle).  Gamma edges (straight,
// with P2 multiplier traces) use the 3-node edge kernels of the Q2 path: the
// midside positions are kept at their edges' midpoints, which makes the
// quadratic edge map the straight one.
//
// Jacobian: the Q2 identities with the geometry's own shape functions, the
// P1 vertex functions M_v with constant gradients h_v: d(det J) = det J h_v,k,
// d(g_a,j) = -g_a,k h_v,j, d(L_ij) = -L_ik h_v,j, d(w) = c0 M_v e_k.
// Quadrature: Radon's 7-point rule (exact to degree 5).
#include <cuda_runtime.h>

#include "viv_internal.h"

namespace viv {
namespace {

constexpr int TEPB = 12;                 // triangles per block
constexpr int TROWS = 21;                // 12 momentum, 3 continuity, 6 pseudo-solid rows
constexpr int TTHREADS = TEPB * TROWS;   // 252
constexpr int TQ = 7;

template <class T>
struct TriTables {
  T N[TQ][6];
  T dN[TQ][6][2];
  T M[TQ][3];
  T W[TQ];
};

// qp record: wdet, g (6 x 2), uw (2), L (4), sigma (00 01 11), inertia (2), div
enum { TQ_WDET = 0, TQ_G = 1, TQ_UW = 13, TQ_L = 15, TQ_SIG = 19, TQ_INERT = 22, TQ_DIV = 24, TQ_REC = 25 };
// element record: current and reference P1 gradients h, h0 (3 x 2), the
// integrated reference weight lame det0 / 2, strain (00 01 11), its trace,
// the current inverse map (00 01 10 11)
enum { TE_H = 0, TE_H0 = 6, TE_WDET0 = 12, TE_EPS = 13, TE_TR = 16, TE_JI = 17, TE_REC = 21 };

template <class T>
__device__ void build_tri_tables(TriTables<T>& tb) {
  if (threadIdx.x >= TQ) return;
  const int q = threadIdx.x;
  const double r = sqrt(15.0);
  const double a = (6.0 - r) / 21.0, b = (6.0 + r) / 21.0;
  const double pts[TQ][2] = {{1.0 / 3.0, 1.0 / 3.0}, {a, a}, {1 - 2 * a, a}, {a, 1 - 2 * a},
                             {b, b}, {1 - 2 * b, b}, {b, 1 - 2 * b}};
  const double wa = (155.0 - r) / 2400.0, wb = (155.0 + r) / 2400.0;
  const double s = pts[q][0], t = pts[q][1];
  const double l[3] = {1 - s - t, s, t};
  const double dl[3][2] = {{-1, -1}, {1, 0}, {0, 1}};
  for (int i = 0; i < 3; ++i) {
    tb.N[q][i] = (T)(l[i] * (2 * l[i] - 1));
    tb.M[q][i] = (T)l[i];
    for (int k = 0; k < 2; ++k) tb.dN[q][i][k] = (T)((4 * l[i] - 1) * dl[i][k]);
  }
  const int ed[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  for (int m = 0; m < 3; ++m) {
    const int i = ed[m][0], j = ed[m][1];
    tb.N[q][3 + m] = (T)(4 * l[i] * l[j]);
    for (int k = 0; k < 2; ++k) tb.dN[q][3 + m][k] = (T)(4 * (l[j] * dl[i][k] + l[i] * dl[j][k]));
  }
  tb.W[q] = (T)(q == 0 ? 9.0 / 80.0 : (q < 4 ? wa : wb));
}

template <class T>
struct TriNodes {
  T u[6][2], ud[6][2];          // velocity and its nodal rate c0 u + hu
  T Xv[3][2], xv[3][2], wv[3][2], p[3];
  T lame;
};

struct TriArgs {
  const int32_t* conn;
  const int32_t* elems;
  int n;
  const double *X, *x, *u, *p, *hu, *hx, *lame;
  const int32_t* node_dof;
  const int32_t* e2nz;
  double rho, mu;
  const double* step;   // device {time, c0}
};

template <class T, bool JAC>
__global__ void __launch_bounds__(TTHREADS) tri_kernel(TriArgs A, double* R, T* vals) {
  __shared__ TriTables<T> tb;
  __shared__ TriNodes<T> en[TEPB];
  __shared__ T qd[TEPB][TQ][TQ_REC];
  __shared__ T ed[TEPB][TE_REC];
  build_tri_tables(tb);
  const int tid = threadIdx.x;
  const double c0d = A.step[1];
  if (tid < TEPB * 16) {   // 16 loader threads per triangle: 6 nodes, 3 vertices, 3 pressures, lame
    const int le = tid / 16, t = tid % 16, gi = blockIdx.x * TEPB + le;
    if (gi < A.n) {
      const int32_t* cn = A.conn + (int64_t)A.elems[gi] * 6;
      TriNodes<T>& E = en[le];
      if (t < 6) {
        const int nd = cn[t];
        for (int i = 0; i < 2; ++i) {
          const double uv = A.u[2 * nd + i];
          E.u[t][i] = (T)uv;
          E.ud[t][i] = (T)(c0d * uv + A.hu[2 * nd + i]);
        }
      } else if (t < 9) {
        const int v = t - 6, nd = cn[v];
        for (int i = 0; i < 2; ++i) {
          const double xv = A.x[2 * nd + i];
          E.Xv[v][i] = (T)A.X[2 * nd + i];
          E.xv[v][i] = (T)xv;
          E.wv[v][i] = (T)(c0d * xv + A.hx[2 * nd + i]);
        }
      } else if (t < 12) {
        E.p[t - 9] = (T)A.p[cn[t - 9]];
      } else if (t == 12) {
        E.lame = (T)A.lame[A.elems[gi]];
      }
    }
  }
  __syncthreads();
  // per triangle: the affine maps, the P1 gradients, the strain (one thread)
  if (tid < TEPB && blockIdx.x * TEPB + tid < A.n) {
    const TriNodes<T>& E = en[tid];
    T* er = ed[tid];
    for (int ref = 0; ref < 2; ++ref) {
      const T(*c)[2] = ref ? E.Xv : E.xv;
      const T J00 = c[1][0] - c[0][0], J01 = c[2][0] - c[0][0];
      const T J10 = c[1][1] - c[0][1], J11 = c[2][1] - c[0][1];
      const T det = J00 * J11 - J01 * J10, id = T(1) / det;
      const T I00 = J11 * id, I01 = -J01 * id, I10 = -J10 * id, I11 = J00 * id;
      const T dl[3][2] = {{-1, -1}, {1, 0}, {0, 1}};
      for (int v = 0; v < 3; ++v) {
        er[(ref ? TE_H0 : TE_H) + 2 * v] = dl[v][0] * I00 + dl[v][1] * I10;
        er[(ref ? TE_H0 : TE_H) + 2 * v + 1] = dl[v][0] * I01 + dl[v][1] * I11;
      }
      if (ref) {
        T wsum = 0;
        for (int q = 0; q < TQ; ++q) wsum += tb.W[q] * det;
        er[TE_WDET0] = wsum * E.lame;
      } else {
        for (int q = 0; q < TQ; ++q) qd[tid][q][TQ_WDET] = tb.W[q] * det;
        er[TE_JI] = I00;
        er[TE_JI + 1] = I01;
        er[TE_JI + 2] = I10;
        er[TE_JI + 3] = I11;
      }
    }
    // the strain of the P1 displacement, constant on the triangle
    T F00 = 0, F01 = 0, F10 = 0, F11 = 0;
    for (int v = 0; v < 3; ++v) {
      const T d0 = E.xv[v][0] - E.Xv[v][0], d1 = E.xv[v][1] - E.Xv[v][1];
      const T h0 = er[TE_H0 + 2 * v], h1 = er[TE_H0 + 2 * v + 1];
      F00 += d0 * h0;
      F01 += d0 * h1;
      F10 += d1 * h0;
      F11 += d1 * h1;
    }
    er[TE_EPS] = F00;
    er[TE_EPS + 1] = T(0.5) * (F01 + F10);
    er[TE_EPS + 2] = F11;
    er[TE_TR] = F00 + F11;
  }
  __syncthreads();
  // per point: gradients, fields, stress (TQ threads per triangle)
  if (tid < TEPB * TQ) {
    const int le = tid / TQ, q = tid % TQ;
    if (blockIdx.x * TEPB + le < A.n) {
      const TriNodes<T>& E = en[le];
      T* Q = qd[le][q];
      const T* er = ed[le];
      const T I00 = er[TE_JI], I01 = er[TE_JI + 1], I10 = er[TE_JI + 2], I11 = er[TE_JI + 3];
      const T mu = (T)A.mu, rho = (T)A.rho;
      T u0 = 0, u1 = 0, ud0 = 0, ud1 = 0, L00 = 0, L01 = 0, L10 = 0, L11 = 0;
      for (int a = 0; a < 6; ++a) {
        const T d0 = tb.dN[q][a][0], d1 = tb.dN[q][a][1];
        const T g0 = d0 * I00 + d1 * I10, g1 = d0 * I01 + d1 * I11;
        Q[TQ_G + 2 * a] = g0;
        Q[TQ_G + 2 * a + 1] = g1;
        const T N = tb.N[q][a];
        u0 += N * E.u[a][0];
        u1 += N * E.u[a][1];
        ud0 += N * E.ud[a][0];
        ud1 += N * E.ud[a][1];
        L00 += E.u[a][0] * g0;
        L01 += E.u[a][0] * g1;
        L10 += E.u[a][1] * g0;
        L11 += E.u[a][1] * g1;
      }
      T w0 = 0, w1 = 0, pq = 0;
      for (int v = 0; v < 3; ++v) {
        w0 += tb.M[q][v] * E.wv[v][0];
        w1 += tb.M[q][v] * E.wv[v][1];
        pq += tb.M[q][v] * E.p[v];
      }
      const T uw0 = u0 - w0, uw1 = u1 - w1;
      Q[TQ_UW] = uw0;
      Q[TQ_UW + 1] = uw1;
      Q[TQ_L] = L00;
      Q[TQ_L + 1] = L01;
      Q[TQ_L + 2] = L10;
      Q[TQ_L + 3] = L11;
      Q[TQ_SIG] = -pq + 2 * mu * L00;
      Q[TQ_SIG + 1] = mu * (L01 + L10);
      Q[TQ_SIG + 2] = -pq + 2 * mu * L11;
      Q[TQ_INERT] = rho * (ud0 + uw0 * L00 + uw1 * L01);
      Q[TQ_INERT + 1] = rho * (ud1 + uw0 * L10 + uw1 * L11);
      Q[TQ_DIV] = L00 + L11;
    }
  }
  __syncthreads();
  int le, t;
  if (tid < 12 * TEPB) {
    le = tid / 12;
    t = tid % 12;
  } else if (tid < 15 * TEPB) {
    le = (tid - 12 * TEPB) / 3;
    t = 12 + (tid - 12 * TEPB) % 3;
  } else {
    le = (tid - 15 * TEPB) / 6;
    t = 15 + (tid - 15 * TEPB) % 6;
  }
  const int gi = blockIdx.x * TEPB + le;
  if (gi >= A.n) return;
  const int e = A.elems[gi];
  const int32_t* cn = A.conn + (int64_t)e * 6;
  const int32_t* nz = A.e2nz + (int64_t)e * TRI_PAIRS;
  const T c0 = (T)c0d, rho = (T)A.rho, mu = (T)A.mu;
  const T* er = ed[le];
  if (t < 12) {  // momentum row (a, i)
    const int a = t >> 1, i = t & 1;
    const int row = A.node_dof[cn[a] * NSLOT + S_UX + i];
    if (row < 0) return;
    if (!JAC) {
      T acc = 0;
      for (int q = 0; q < TQ; ++q) {
        const T* Q = qd[le][q];
        const T ga0 = Q[TQ_G + 2 * a], ga1 = Q[TQ_G + 2 * a + 1];
        const T s0 = i == 0 ? Q[TQ_SIG] : Q[TQ_SIG + 1];
        const T s1 = i == 0 ? Q[TQ_SIG + 1] : Q[TQ_SIG + 2];
        acc += Q[TQ_WDET] * (tb.N[q][a] * Q[TQ_INERT + i] + ga0 * s0 + ga1 * s1);
      }
      R[row] += (double)acc;
      return;
    }
    // u columns of the 6 nodes
    for (int b = 0; b < 6; ++b) {
      T au[2] = {0, 0};
      for (int q = 0; q < TQ; ++q) {
        const T* Q = qd[le][q];
        const T Na = tb.N[q][a], Nb = tb.N[q][b];
        const T ga0 = Q[TQ_G + 2 * a], ga1 = Q[TQ_G + 2 * a + 1];
        const T gb0 = Q[TQ_G + 2 * b], gb1 = Q[TQ_G + 2 * b + 1];
        const T uwg = Q[TQ_UW] * gb0 + Q[TQ_UW + 1] * gb1;
        const T gagb = ga0 * gb0 + ga1 * gb1;
        const T gbi = i == 0 ? gb0 : gb1;
        for (int k = 0; k < 2; ++k) {
          const T Lik = Q[TQ_L + 2 * i + k], gak = k == 0 ? ga0 : ga1;
          T v = rho * Na * Nb * Lik + mu * gak * gbi;
          if (k == i) v += rho * Na * (c0 * Nb + uwg) + mu * gagb;
          au[k] += Q[TQ_WDET] * v;
        }
      }
      for (int k = 0; k < 2; ++k) {
        const int s = nz[tpairA(a, i, 2 * b + k)];
        if (s >= 0) vals[s] += au[k];
      }
    }
    // position columns of the 3 vertices (shape derivatives with the P1 gradients h_v)
    for (int v = 0; v < 3; ++v) {
      const T hv0 = er[TE_H + 2 * v], hv1 = er[TE_H + 2 * v + 1];
      T ax[2] = {0, 0};
      for (int q = 0; q < TQ; ++q) {
        const T* Q = qd[le][q];
        const T Na = tb.N[q][a], Mv = tb.M[q][v];
        const T ga0 = Q[TQ_G + 2 * a], ga1 = Q[TQ_G + 2 * a + 1];
        const T si0 = i == 0 ? Q[TQ_SIG] : Q[TQ_SIG + 1];
        const T si1 = i == 0 ? Q[TQ_SIG + 1] : Q[TQ_SIG + 2];
        const T uwh = Q[TQ_UW] * hv0 + Q[TQ_UW + 1] * hv1;
        const T gah = ga0 * hv0 + ga1 * hv1;
        const T hvi = i == 0 ? hv0 : hv1;
        const T sig_h = si0 * hv0 + si1 * hv1;
        const T rai = Na * Q[TQ_INERT + i] + ga0 * si0 + ga1 * si1;
        const T cm = c0 * Mv + uwh;
        for (int k = 0; k < 2; ++k) {
          const T Lik = Q[TQ_L + 2 * i + k], gak = k == 0 ? ga0 : ga1, hvk = k == 0 ? hv0 : hv1;
          const T gaLk = ga0 * Q[TQ_L + k] + ga1 * Q[TQ_L + 2 + k];
          ax[k] += Q[TQ_WDET] * (-rho * Na * Lik * cm - gak * sig_h - mu * (Lik * gah + hvi * gaLk) + rai * hvk);
        }
      }
      for (int k = 0; k < 2; ++k) {
        const int s = nz[tpairA(a, i, 12 + 2 * v + k)];
        if (s >= 0) vals[s] += ax[k];
      }
    }
    for (int c = 0; c < 3; ++c) {
      T acc = 0;
      for (int q = 0; q < TQ; ++q) acc -= qd[le][q][TQ_WDET] * qd[le][q][TQ_G + 2 * a + i] * tb.M[q][c];
      const int s = nz[tpairA(a, i, 18 + c)];
      if (s >= 0) vals[s] += acc;
    }
  } else if (t < 15) {  // continuity row c
    const int c = t - 12;
    const int row = A.node_dof[cn[c] * NSLOT + S_P];
    if (row < 0) return;
    if (!JAC) {
      T acc = 0;
      for (int q = 0; q < TQ; ++q) acc -= qd[le][q][TQ_WDET] * tb.M[q][c] * qd[le][q][TQ_DIV];
      R[row] += (double)acc;
      return;
    }
    for (int b = 0; b < 6; ++b) {
      T au[2] = {0, 0};
      for (int q = 0; q < TQ; ++q) {
        const T wm = qd[le][q][TQ_WDET] * tb.M[q][c];
        au[0] -= wm * qd[le][q][TQ_G + 2 * b];
        au[1] -= wm * qd[le][q][TQ_G + 2 * b + 1];
      }
      for (int k = 0; k < 2; ++k) {
        const int s = nz[tpairB(c, 2 * b + k)];
        if (s >= 0) vals[s] += au[k];
      }
    }
    for (int v = 0; v < 3; ++v) {
      const T hv0 = er[TE_H + 2 * v], hv1 = er[TE_H + 2 * v + 1];
      T ax[2] = {0, 0};
      for (int q = 0; q < TQ; ++q) {
        const T* Q = qd[le][q];
        const T wm = Q[TQ_WDET] * tb.M[q][c];
        for (int k = 0; k < 2; ++k) {
          const T hvk = k == 0 ? hv0 : hv1;
          const T Lh = Q[TQ_L + k] * hv0 + Q[TQ_L + 2 + k] * hv1;   // sum_i L_ik h_v,i
          ax[k] += wm * (Lh - Q[TQ_DIV] * hvk);
        }
      }
      for (int k = 0; k < 2; ++k) {
        const int s = nz[tpairB(c, 12 + 2 * v + k)];
        if (s >= 0) vals[s] += ax[k];
      }
    }
  } else {  // pseudo-solid row (v, i)
    const int r = t - 15;
    const int v = r >> 1, i = r & 1;
    const int row = A.node_dof[cn[v] * NSLOT + S_XX + i];
    if (row < 0) return;
    const T h0 = er[TE_H0 + 2 * v], h1 = er[TE_H0 + 2 * v + 1];
    if (!JAC) {
      const T hi = i == 0 ? h0 : h1;
      const T e0 = i == 0 ? er[TE_EPS] : er[TE_EPS + 1];
      const T e1 = i == 0 ? er[TE_EPS + 1] : er[TE_EPS + 2];
      R[row] += (double)(er[TE_WDET0] * (hi * er[TE_TR] + 2 * (h0 * e0 + h1 * e1)));
      return;
    }
    for (int w = 0; w < 3; ++w) {
      const T k0 = er[TE_H0 + 2 * w], k1 = er[TE_H0 + 2 * w + 1];
      const T hi = i == 0 ? h0 : h1, kwi = i == 0 ? k0 : k1;
      for (int k = 0; k < 2; ++k) {
        const T hk = k == 0 ? h0 : h1, kwk = k == 0 ? k0 : k1;
        T val = hi * kwk + hk * kwi;
        if (k == i) val += h0 * k0 + h1 * k1;
        const int s = nz[tpairC(v, i, w, k)];
        if (s >= 0) vals[s] += er[TE_WDET0] * val;
      }
    }
  }
}

__global__ void tri_area_kernel(const int32_t* conn, const double* X, int64_t E, double* area) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int32_t* c = conn + e * 6;
  const double J00 = X[2 * c[1]] - X[2 * c[0]], J01 = X[2 * c[2]] - X[2 * c[0]];
  const double J10 = X[2 * c[1] + 1] - X[2 * c[0] + 1], J11 = X[2 * c[2] + 1] - X[2 * c[0] + 1];
  area[e] = 0.5 * (J00 * J11 - J01 * J10);
}

// a midside node's position: the midpoint of its edge's end vertices (the P1
// position field there); Gamma midpoints follow delta like their vertices
__global__ void midside_kernel(int64_t n, const int32_t* mid_parent, const int32_t* tags, double* x) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n) return;
  const int32_t va = mid_parent[2 * a], vb = mid_parent[2 * a + 1];
  if (va < 0 || (tags[a] & VIV_TAG_CYL)) return;
  x[2 * a] = 0.5 * (x[2 * va] + x[2 * vb]);
  x[2 * a + 1] = 0.5 * (x[2 * va + 1] + x[2 * vb + 1]);
}

}  // namespace

void launch_triangle_areas(const Mesh& m, double* area, cudaStream_t s) {
  Launched L(K_VEC, s);
  tri_area_kernel<<<(unsigned)((m.n_elems + 127) / 128), 128, 0, s>>>(m.d_conn, m.d_X, m.n_elems, area);
  VIV_CUDA(cudaGetLastError());
}

void launch_midside_positions(const Mesh& m, double* x, cudaStream_t s) {
  Launched L(K_VEC, s);
  midside_kernel<<<(unsigned)((m.n_nodes + 255) / 256), 256, 0, s>>>(m.n_nodes, m.d_mid_parent, m.d_tags, x);
  VIV_CUDA(cudaGetLastError());
}

template <class T, bool JAC>
void run_assembly_tri(const Mesh& m, const CaseState& st, const vivParams& prm, double* R, T* vals, cudaStream_t s) {
  TriArgs A;
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
  A.step = st.step;
  for (int c = 0; c + 1 < (int)m.color_off.size(); ++c) {
    A.elems = m.d_color_elems + m.color_off[c];
    A.n = m.color_off[c + 1] - m.color_off[c];
    if (!A.n) continue;
    Launched L(JAC ? K_JAC : K_RES, s);
    tri_kernel<T, JAC><<<(A.n + TEPB - 1) / TEPB, TTHREADS, 0, s>>>(A, R, vals);
  }
  VIV_CUDA(cudaGetLastError());
}

template void run_assembly_tri<double, false>(const Mesh&, const CaseState&, const vivParams&, double*, double*,
                                              cudaStream_t);
template void run_assembly_tri<double, true>(const Mesh&, const CaseState&, const vivParams&, double*, double*,
                                             cudaStream_t);
template void run_assembly_tri<float, true>(const Mesh&, const CaseState&, const vivParams&, double*, float*,
                                            cudaStream_t);

}  // namespace viv
