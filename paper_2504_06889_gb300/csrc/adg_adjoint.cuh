// Discrete adjoint of the ADER-DG step for linear acoustics with a per-cell wave speed c
// (K = rho c^2).  For a fixed dt the step Q^{n+1} = S(c) Q^n is linear; the adjoint state
// lam^n = S^T lam^{n+1} is obtained by transposing, in reverse order, the surface update, the
// Rusanov flux (whose face speed s = max(c-, c+) enters as a constant for lam), the face
// extrapolation, the volume integral, the time average and the Picard sweeps
// q^r = Q - dt P R(q^{r-1}).  The material gradient per cell has two parts:
//  - through the fluxes: <lam^{n+1}, dS/dK_c Q^n>, evaluated by a tangent-linear pass of the cell's
//    predictor (q, dq/dK_c) -- no Picard iterates are stored;
//  - through the face speed: s = max(c-, c+) changes with the larger of the two speeds;
//    dG/ds = (q- - q+)/2 (half to each side on a tie).
// dt is that of the forward run, held fixed (it depends on max c only).
#pragma once

#include "adg_kernels.cuh"

namespace adg {

struct AdjArgs {
  StepArgs s;          // mesh, tables, PDE; s.Q = forward state Q^n, s.traces = its FP64 traces
  double* lam;         // adjoint state: dJ/dQ^{n+1} on entry, dJ/dQ^n on exit
  double* padj;        // projections of lam onto the faces [cell][dir][side][v][j]
  double* gK;          // dJ/dK per cell (accumulated)
  double* gS;          // dJ/dc per cell through the Rusanov face speed (accumulated)
  double dt;
};

// P_side(dir, v, j) = sum_a psi_side(a) / (h_dir w_a) lam(node(dir, j, a), v)
template <class C>
__global__ void k_adj_trace(const __grid_constant__ AdjArgs a) {
  constexpr int n = C::n, V = C::V, D = C::D, NS = C::NS, NF = C::NF;
  const size_t total = (size_t)a.s.ncells * D * 2 * V * NF;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(g % NF);
    const int v = (int)((g / NF) % V);
    const int side = (int)((g / ((size_t)NF * V)) % 2);
    const int dir = (int)((g / ((size_t)NF * V * 2)) % D);
    const int cell = (int)(g / ((size_t)NF * V * 2 * D));
    const double* lc = a.lam + (size_t)cell * V * NS + (size_t)v * NS;
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const double psi = side ? a.s.tab.psi1[m] : a.s.tab.psi0[m];
      s += psi / a.s.tab.w[m] * lc[node_of_face<D, n>(dir, j, m)];
    }
    a.padj[g] = s * a.s.invh[dir];
  }
}

template <class C> struct AdjSmem {
  static constexpr int PD = Pencil<C>::PER_DIR;
  // lam of the cell (FP64) + two pencil-layout buffers (value and tangent) of D x V entries
  static constexpr size_t lam = sizeof(double) * C::CPB * C::V * C::NS;
  static constexpr size_t pen = sizeof(double) * C::CPB * 2 * C::D * C::V * PD;
  static constexpr size_t red = sizeof(double) * 2 * C::CPB * 32;
  static constexpr size_t total = lam + pen + red;
};

// One thread per node.  T: arithmetic of the tangent and transposed Picard sweeps.
template <class C, class T>
__global__ void __launch_bounds__(C::THREADS) k_adj_cell(const __grid_constant__ AdjArgs a) {
  static_assert(C::PDE == 0, "the adjoint is built for linear acoustics");
  constexpr int n = C::n, V = C::V, D = C::D, NS = C::NS, NF = C::NF, CPB = C::CPB;
  constexpr int S = Pencil<C>::S, PD = Pencil<C>::PER_DIR;
  extern __shared__ __align__(16) unsigned char adj_smem[];
  const StepArgs& st = a.s;
  const int lc = threadIdx.x / NS, i = threadIdx.x % NS;
  const int cell = blockIdx.x * CPB + lc;
  const bool valid = cell < st.ncells;
  const int cl = valid ? cell : 0;
  const double dt = a.dt;
  const double rho = st.pp.rho, irho = st.pp.irho;
  auto cspeed = [&](int c) { return st.pp.cell_c ? fabs(st.pp.cell_c[c]) : st.pp.c; };
  const double cc = cspeed(cl);
  const double K = rho * cc * cc;

  double* sLam = reinterpret_cast<double*>(adj_smem) + (size_t)lc * V * NS;
  double* sPen = reinterpret_cast<double*>(adj_smem + AdjSmem<C>::lam) + (size_t)lc * 2 * D * V * PD;
  double* sRed = reinterpret_cast<double*>(adj_smem + AdjSmem<C>::lam + AdjSmem<C>::pen);
  T* sA = reinterpret_cast<T*>(sPen);                // value pencils
  T* sB = sA + (size_t)D * V * PD;                   // tangent pencils

  const int idx[3] = {i % n, (i / n) % n, i / (n * n)};
  int pb[3], jf[3];
  pb[0] = (i / n) * S;
  if (D == 2) {
    pb[1] = idx[0] * S;
    pb[2] = 0;
    jf[0] = idx[1];
    jf[1] = idx[0];
    jf[2] = 0;
  } else {
    pb[1] = (idx[0] + n * idx[2]) * S;
    pb[2] = (idx[0] + n * idx[1]) * S;
    jf[0] = idx[1] + n * idx[2];
    jf[1] = idx[0] + n * idx[2];
    jf[2] = idx[0] + n * idx[1];
  }
  const double* lamc = a.lam + (size_t)cl * V * NS;
  double lamv[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    lamv[v] = lamc[v * NS + i];
    sLam[v * NS + i] = lamv[v];
  }
  // zero the pencil pads (read by nothing, but keep the buffer clean)
  __syncthreads();

  // ---- phase A: adjoints of the time-averaged state (traces) and flux (traces + volume) ---------
  double lQ[V], lF[D][V], gS_loc = 0.0;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    lQ[v] = 0.0;
#pragma unroll
    for (int dir = 0; dir < D; ++dir) lF[dir][v] = 0.0;
  }
  constexpr size_t tcell = (size_t)D * 2 * 2 * V * NF;  // forward traces per cell
  constexpr size_t pcell = (size_t)D * 2 * V * NF;      // adjoint projections per cell
  const double* TQ = reinterpret_cast<const double*>(st.traces);
#pragma unroll
  for (int dir = 0; dir < D; ++dir) {
    const int cln = neighbour(st, cl, dir, 0), crn = neighbour(st, cl, dir, 1);
    const double cm = cspeed(cln), cp = cspeed(crn);
    const double sR = fmax(cc, cp), sL = fmax(cm, cc);
    const int a_ = idx[dir], j = jf[dir];
    const double p1 = st.tab.psi1[a_], p0 = st.tab.psi0[a_];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      // face adjoints: dJ/dG on the right (c | cr) and left (cl | c) faces
      const double gR = dt * (-a.padj[(size_t)cl * pcell + ((dir * 2 + 1) * V + v) * NF + j] +
                              a.padj[(size_t)crn * pcell + ((dir * 2 + 0) * V + v) * NF + j]);
      const double gL = dt * (-a.padj[(size_t)cln * pcell + ((dir * 2 + 1) * V + v) * NF + j] +
                              a.padj[(size_t)cl * pcell + ((dir * 2 + 0) * V + v) * NF + j]);
      // G = (F- + F+)/2 + s/2 (q- - q+); this cell is "-" on the right face, "+" on the left
      lQ[v] += p1 * 0.5 * sR * gR - p0 * 0.5 * sL * gL;
      lF[dir][v] += p1 * 0.5 * gR + p0 * 0.5 * gL;
      // face speed: counted once per face node (by the node with a = 0), owned by the larger c
      if (a_ == 0) {
        const double qmR = TQ[(size_t)cl * tcell + (((dir * 2 + 1) * 2 + 0) * V + v) * NF + j];
        const double qpR = TQ[(size_t)crn * tcell + (((dir * 2 + 0) * 2 + 0) * V + v) * NF + j];
        const double qmL = TQ[(size_t)cln * tcell + (((dir * 2 + 1) * 2 + 0) * V + v) * NF + j];
        const double qpL = TQ[(size_t)cl * tcell + (((dir * 2 + 0) * 2 + 0) * V + v) * NF + j];
        const double wR = cc > cp ? 1.0 : (cc == cp ? 0.5 : 0.0);
        const double wL = cc > cm ? 1.0 : (cc == cm ? 0.5 : 0.0);
        gS_loc += wR * gR * 0.5 * (qmR - qpR) + wL * gL * 0.5 * (qmL - qpL);
      }
      // volume: Q_m += dt/h sum_dir (1/w_{m_dir}) sum_a w_a D[a][m_dir] Fbar(m[dir<-a])
      double sv = 0.0;
#pragma unroll
      for (int m = 0; m < n; ++m)
        sv += st.tab.D[a_][m] / st.tab.w[m] * sLam[v * NS + node_of_face<D, n>(dir, jf[dir], m)];
      lF[dir][v] += dt * st.invh[dir] * st.tab.w[a_] * sv;
    }
  }
  double lQt[V];  // adjoint of Qbar including the flux: Fbar = A Qbar
#pragma unroll
  for (int v = 0; v < V; ++v) lQt[v] = lQ[v];
#pragma unroll
  for (int dir = 0; dir < D; ++dir) {
    lQt[1 + dir] += K * lF[dir][0];
    lQt[0] += irho * lF[dir][1 + dir];
  }

  // ---- phase B: tangent of the predictor w.r.t. K (gradient through the fluxes) ----------------
  T Qh[V];
#pragma unroll
  for (int v = 0; v < V; ++v) Qh[v] = (T)st.Q[((size_t)cl * V + v) * NS + i];
  T Dr[D][n];
#pragma unroll
  for (int dir = 0; dir < D; ++dir)
#pragma unroll
    for (int m = 0; m < n; ++m) Dr[dir][m] = (T)(st.tab.D[idx[dir]][m] * st.invh[dir]);
  const T Kt = (T)K, irt = (T)irho;
  double gK_loc = 0.0;
  {
    T q[n][V], dq[n][V];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        q[k][v] = Qh[v];
        dq[k][v] = T(0);
      }
    for (int r = 0; r < st.picard_iters; ++r) {
      T qn[n][V], dqn[n][V];
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          qn[k][v] = Qh[v];
          dqn[k][v] = T(0);
        }
#pragma unroll
      for (int k = 0; k < n; ++k) {
        // F_dir = (K v_dir, p / rho e_dir);  dF_dir/dK_c applied: K dv_dir + v_dir in the p row
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
          sA[(dir * V + 0) * PD + pb[dir] + idx[dir]] = Kt * q[k][1 + dir];
          sA[(dir * V + 1 + dir) * PD + pb[dir] + idx[dir]] = q[k][0] * irt;
          sB[(dir * V + 0) * PD + pb[dir] + idx[dir]] = Kt * dq[k][1 + dir] + q[k][1 + dir];
          sB[(dir * V + 1 + dir) * PD + pb[dir] + idx[dir]] = dq[k][0] * irt;
        }
        __syncthreads();
        T rv[V], drv[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          rv[v] = T(0);
          drv[v] = T(0);
        }
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
#pragma unroll
          for (int vv = 0; vv < 2; ++vv) {
            const int v = vv == 0 ? 0 : 1 + dir;
            const T* fa = sA + (dir * V + v) * PD + pb[dir];
            const T* fb = sB + (dir * V + v) * PD + pb[dir];
#pragma unroll
            for (int m = 0; m < n; ++m) {
              rv[v] += Dr[dir][m] * fa[m];
              drv[v] += Dr[dir][m] * fb[m];
            }
          }
        }
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int kk = 0; kk < n; ++kk) {
            const T c = (T)(dt * st.tab.P[kk][k]);
            qn[kk][v] -= c * rv[v];
            dqn[kk][v] -= c * drv[v];
          }
        __syncthreads();
      }
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          q[k][v] = qn[k][v];
          dq[k][v] = dqn[k][v];
        }
    }
    // Qbar, dQbar/dK; dFbar = A dQbar + (v_dir in the p row)
    double Qb[V], dQb[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      Qb[v] = 0.0;
      dQb[v] = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) {
        Qb[v] += st.tab.w[k] * (double)q[k][v];
        dQb[v] += st.tab.w[k] * (double)dq[k][v];
      }
    }
    // <lF, A_K Qbar> + <lQt, dQbar>
#pragma unroll
    for (int dir = 0; dir < D; ++dir) gK_loc += lF[dir][0] * Qb[1 + dir];
#pragma unroll
    for (int v = 0; v < V; ++v) gK_loc += lQt[v] * dQb[v];
  }

  // ---- phase C: transposed Picard sweeps -> dJ/dQ^n ------------------------------------------
  double lQhat[V];
#pragma unroll
  for (int v = 0; v < V; ++v) lQhat[v] = 0.0;
  {
    T mu[n][V];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < V; ++v) mu[k][v] = (T)(st.tab.w[k] * lQt[v]);
    for (int r = 0; r < st.picard_iters; ++r) {
      // q^r = Q 1 - dt P R(q^{r-1}):  lam_Q += sum_k mu_k;  nu_l = -dt sum_k P[k][l] mu_k
      T nu[n][V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) s += (double)mu[k][v];
        lQhat[v] += s;
#pragma unroll
        for (int l = 0; l < n; ++l) {
          T t = T(0);
#pragma unroll
          for (int k = 0; k < n; ++k) t += (T)(st.tab.P[k][l]) * mu[k][v];
          nu[l][v] = (T)(-dt) * t;
        }
      }
      // mu^{r-1} = R^T nu: R = sum_dir (1/h) D_dir A_dir; per slice l, A^T nu to the pencils,
      // then the contraction with D^T along each direction
#pragma unroll
      for (int l = 0; l < n; ++l) {
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
          sA[(dir * V + 0) * PD + pb[dir] + idx[dir]] = nu[l][1 + dir] * irt;  // (A^T nu)_p
          sA[(dir * V + 1 + dir) * PD + pb[dir] + idx[dir]] = Kt * nu[l][0];    // (A^T nu)_{v_dir}
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < V; ++v) mu[l][v] = T(0);
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
#pragma unroll
          for (int vv = 0; vv < 2; ++vv) {
            const int v = vv == 0 ? 0 : 1 + dir;
            const T* fa = sA + (dir * V + v) * PD + pb[dir];
            T s = T(0);
#pragma unroll
            for (int m = 0; m < n; ++m) s += (T)(st.tab.D[m][idx[dir]] * st.invh[dir]) * fa[m];
            mu[l][v] += s;
          }
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int k = 0; k < n; ++k) lQhat[v] += (double)mu[k][v];
  }

  // ---- outputs: lam^n = lam^{n+1} + predictor part; gradients reduced per cell ----------------
  if (valid) {
    double* lw = a.lam + (size_t)cell * V * NS;
#pragma unroll
    for (int v = 0; v < V; ++v) lw[v * NS + i] = lamv[v] + lQhat[v];
  }
  // block reduction per cell, fixed order (deterministic)
  double* rk = sRed + (size_t)lc * 64;
  if (i < 64) {
    rk[i] = 0.0;
  }
  __syncthreads();
  // tree over the NS nodes of the cell: stage through shared memory
  double* red = sLam;  // reuse: V*NS >= 2*NS
  red[i] = gK_loc;
  red[NS + i] = gS_loc;
  __syncthreads();
  if (i == 0 && valid) {
    double sk = 0.0, ss = 0.0;
    for (int t = 0; t < NS; ++t) {
      sk += red[t];
      ss += red[NS + t];
    }
    a.gK[cell] += sk;
    a.gS[cell] += ss;
  }
}

template <class C>
cudaError_t launch_adj_trace(const AdjArgs& a, cudaStream_t s) {
  const size_t total = (size_t)a.s.ncells * C::D * 2 * C::V * C::NF;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_adj_trace<C><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <class C, class T>
cudaError_t launch_adj_cell(const AdjArgs& a, cudaStream_t s) {
  const size_t smem = AdjSmem<C>::total;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_adj_cell<C, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int blocks = (a.s.ncells + C::CPB - 1) / C::CPB;
  k_adj_cell<C, T><<<blocks, C::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

using AdjFn = cudaError_t (*)(const AdjArgs&, cudaStream_t);

}  // namespace adg
