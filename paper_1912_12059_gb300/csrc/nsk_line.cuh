// nsk_line.cuh -- line-per-thread stage kernels of the FP32 operator for 3D elements with N = 3
// (4 x 4 x 4 nodes), stage schedule fused_face = 4.
//
// The BR1 lifting and the volume + update kernel of the separate face schedule, with 16 threads
// per element instead of 64: thread t = j + 4 kk owns the line of nodes (0..3, j, kk) in direction
// x, i.e. the contiguous nodes 4t .. 4t + 3. Its nodal values move with 16-byte loads and stores,
// the contractions along x run in registers, and those along y and z read the other threads'
// lines from shared memory, 16 bytes at a time. Index arithmetic is per line instead of per node.
// The kernels read and write the same arrays in the same layouts as k_lift and k_volume (so the
// face kernel between them is unchanged) and evaluate every value with the same operations in the
// same order, so the results are the same bit for bit.
#pragma once

namespace nsk {

namespace line {
constexpr int NPE = 64, NFN = 16, NF = 6, NV = 5, NW = 4, NVF = 9;
// shared memory per element (floats)
constexpr int kLiftElem = NW * NPE + 4 * NW * NFN;  // sw and sws; sfv (y, z: 2 NW NPE) reuses both
constexpr int kVolElem = NF * NV * NFN + 2 * NV * NPE;            // sfs, sfy, sfz
}  // namespace line

template <int G>
__host__ __device__ constexpr int lift_line_smem() {
  return G * line::kLiftElem + tab_smem<3, 4>();
}
template <int G>
__host__ __device__ constexpr int volume_line_smem() {
  return G * line::kVolElem + tab_smem<3, 4>() + 2;
}

__device__ __forceinline__ float f4_at(const float4& a, int i) {
  return i == 0 ? a.x : (i == 1 ? a.y : (i == 2 ? a.z : a.w));
}
__device__ __forceinline__ float4 f4_make(const float (&a)[4]) { return make_float4(a[0], a[1], a[2], a[3]); }

// BR1 lifting of lift_group (model II, viscous form stored), line per thread.
// resident blocks asked of the compiler: 128-thread blocks 7 (at most 72 registers), 256-thread
// blocks 3 (at most 85)
template <int G>
__host__ __device__ constexpr int lift_line_min_blocks() {
  return G * 16 <= 128 ? 7 : 3;
}

template <int G>
__global__ void __launch_bounds__(G * 16, lift_line_min_blocks<G>())
    k_lift_line(const NskParams p, const float* __restrict__ U, const float* __restrict__ Utr,
                float* __restrict__ Q, float* __restrict__ FVtr, int* __restrict__ err) {
  using R = float;
  using namespace line;
  extern __shared__ __align__(16) unsigned char line_smem_raw[];
  R* sm = reinterpret_cast<R*>(line_smem_raw);
  const int le = threadIdx.x >> 4, t = threadIdx.x & 15, j = t & 3, kk = t >> 2;
  R* sw = sm + le * kLiftElem;      // [w][node] primitive variables
  R* sws = sw + NW * NPE;            // [slot - 2][w][fn] 2 w* on the y and z faces
  R* sfv = sw;                       // [k - 1][c][node] F^v_k, once sw and sws have been read
  R* tb = sm + G * kLiftElem;
  const auto& T = TabSel<R>::get(p);
  const int e = (int)blockIdx.x * G + le;
  const bool valid = e < p.E;
  const size_t nn = (size_t)p.nne, pl = (size_t)NF * p.nfe;
  const int g0 = e * NPE + 4 * t;
  int eflag = 0;
  stage_tables<R, 3, 4>(T, tb, R(1), R(0.5));

  R w[NW][4], wsx[2][NW];
  ElemIdx ex{};
  if (valid) {
    ex = elem_idx<3>(p, e);
    float4 uv[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) uv[v] = *reinterpret_cast<const float4*>(U + v * nn + g0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // lift_store_w
      const R rho = f4_at(uv[0], i);
      eflag |= rho_flags(rho);
      const R inv = rcp_s(rho);
#pragma unroll
      for (int a = 0; a < 3; ++a) w[a][i] = f4_at(uv[1 + a], i) * inv;
      w[3][i] = f4_at(uv[4], i);
    }
#pragma unroll
    for (int c = 0; c < NW; ++c) *reinterpret_cast<float4*>(sw + c * NPE + 4 * t) = f4_make(w[c]);
    // 2 w* on the x faces at face node t: kept in registers
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int en = nbr_of(p, ex, 0, s ? 1 : -1);
      const R* to = Utr + (size_t)s * p.nfe + (e * NFN + t);
      const R* tn = Utr + (size_t)(1 - s) * p.nfe + (en * NFN + t);
      R uo[NV], un[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        uo[v] = to[v * pl];
        un[v] = tn[v * pl];
      }
      lift_wstar<R, 3, 1, NV>(uo, un, wsx[s], eflag);
    }
    // 2 w* on four face nodes of a y or z face (one task per thread), to shared memory
    {
      const int slot = 2 + (t >> 2), k = slot >> 1, s = slot & 1, fnb = 4 * (t & 3);
      const int en = nbr_of(p, ex, k, s ? 1 : -1);
      const R* to = Utr + (size_t)slot * p.nfe + (e * NFN + fnb);
      const R* tn = Utr + (size_t)(2 * k + 1 - s) * p.nfe + (en * NFN + fnb);
      float4 uo4[NV], un4[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        uo4[v] = *reinterpret_cast<const float4*>(to + v * pl);
        un4[v] = *reinterpret_cast<const float4*>(tn + v * pl);
      }
      R ws4[NW][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        R uo[NV], un[NV], ws1[NW];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          uo[v] = f4_at(uo4[v], i);
          un[v] = f4_at(un4[v], i);
        }
        lift_wstar<R, 3, 1, NV>(uo, un, ws1, eflag);
#pragma unroll
        for (int c = 0; c < NW; ++c) ws4[c][i] = ws1[c];
      }
#pragma unroll
      for (int c = 0; c < NW; ++c)
        *reinterpret_cast<float4*>(sws + (slot - 2) * (NW * NFN) + c * NFN + fnb) = f4_make(ws4[c]);
    }
  }
  __syncthreads();

  // lift_q per node, direction by direction: q[i][k NW + c]
  R q[4][12], fy[NW][4], fz[NW][4];  // fy, fz: the viscous flux F^v_y, F^v_z at the line's nodes
  if (valid) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // x: the thread's own line
      R dk[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) dk[jj] = tb[i * 4 + jj];
      const R lpk = tb[48 + i], lmk = tb[60 + i];
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        R vol = 0;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) vol = fmaf(dk[jj], w[c][jj], vol);
        q[i][c] = fmaf(wsx[1][c], lpk, fmaf(-wsx[0][c], lmk, -vol));
      }
    }
    {  // y: lines (jj, kk), face nodes i + 4 kk
      R dk[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) dk[jj] = tb[(4 + j) * 4 + jj];
      const R lpk = tb[48 + 4 + j], lmk = tb[60 + 4 + j];
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        float4 ln[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) ln[jj] = *reinterpret_cast<const float4*>(sw + c * NPE + 4 * (jj + 4 * kk));
        const float4 wp = *reinterpret_cast<const float4*>(sws + 1 * (NW * NFN) + c * NFN + 4 * kk);
        const float4 wm = *reinterpret_cast<const float4*>(sws + 0 * (NW * NFN) + c * NFN + 4 * kk);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          R vol = 0;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) vol = fmaf(dk[jj], f4_at(ln[jj], i), vol);
          q[i][NW + c] = fmaf(f4_at(wp, i), lpk, fmaf(-f4_at(wm, i), lmk, -vol));
        }
      }
    }
    {  // z: lines (j, ll), face nodes i + 4 j
      R dk[4];
#pragma unroll
      for (int ll = 0; ll < 4; ++ll) dk[ll] = tb[(8 + kk) * 4 + ll];
      const R lpk = tb[48 + 8 + kk], lmk = tb[60 + 8 + kk];
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        float4 ln[4];
#pragma unroll
        for (int ll = 0; ll < 4; ++ll) ln[ll] = *reinterpret_cast<const float4*>(sw + c * NPE + 4 * (j + 4 * ll));
        const float4 wp = *reinterpret_cast<const float4*>(sws + 3 * (NW * NFN) + c * NFN + 4 * j);
        const float4 wm = *reinterpret_cast<const float4*>(sws + 2 * (NW * NFN) + c * NFN + 4 * j);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          R vol = 0;
#pragma unroll
          for (int ll = 0; ll < 4; ++ll) vol = fmaf(dk[ll], f4_at(ln[ll], i), vol);
          q[i][2 * NW + c] = fmaf(f4_at(wp, i), lpk, fmaf(-f4_at(wm, i), lmk, -vol));
        }
      }
    }
    // the viscous form (visc_of, visc_store) and the viscous flux F^v_k = (tau_{k.}, grad_k c)
    R qf[NVF][4], fx[NW][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      R tau[3][3], gc[3];
      visc_of<R, 3>(q[i], tau, gc);
      int c = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = k; a < 3; ++a) qf[c++][i] = tau[k][a];
#pragma unroll
      for (int k = 0; k < 3; ++k) qf[c++][i] = gc[k];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        fx[a][i] = tau[0][a];
        fy[a][i] = tau[1][a];
        fz[a][i] = tau[2][a];
      }
      fx[3][i] = gc[0];
      fy[3][i] = gc[1];
      fz[3][i] = gc[2];
    }
#pragma unroll
    for (int c = 0; c < NVF; ++c) *reinterpret_cast<float4*>(Q + c * nn + g0) = f4_make(qf[c]);
    // x faces (slots 0, 1) at face node t: traces along the thread's own line
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const R* Lmu = s ? T.lpmu : T.lmmu;
      const R* Lkb = s ? T.lpkb : T.lmkb;
      R* o = FVtr + (size_t)s * p.nfe + (e * NFN + t);
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        const R* L = c < 3 ? Lmu : Lkb;
        R acc = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) acc = fmaf(L[i], fx[c][i], acc);
        o[c * pl] = acc;
      }
    }
  }
  __syncthreads();  // sw and sws are read: sfv takes their place
  if (valid) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      *reinterpret_cast<float4*>(sfv + 0 * (NW * NPE) + c * NPE + 4 * t) = f4_make(fy[c]);
      *reinterpret_cast<float4*>(sfv + 1 * (NW * NPE) + c * NPE + 4 * t) = f4_make(fz[c]);
    }
  }
  __syncthreads();
  if (valid) {  // y and z faces: four face nodes of one slot per thread
    const int slot = 2 + (t >> 2), k = slot >> 1, s = slot & 1, g = t & 3;
    const R* Lmu = s ? T.lpmu : T.lmmu;
    const R* Lkb = s ? T.lpkb : T.lmkb;
    R* o = FVtr + (size_t)slot * p.nfe + (e * NFN + 4 * g);
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      const R* L = c < 3 ? Lmu : Lkb;
      const R* f = sfv + (k - 1) * (NW * NPE) + c * NPE;
      R acc[4] = {0, 0, 0, 0};
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        // k = 1: line node (i, jj, g); k = 2: line node (i, g, jj)
        const float4 ln = *reinterpret_cast<const float4*>(f + 4 * (k == 1 ? jj + 4 * g : g + 4 * jj));
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = fmaf(L[jj], f4_at(ln, i), acc[i]);
      }
      *reinterpret_cast<float4*>(o + c * pl) = f4_make(acc);
    }
  }
  if (eflag) atomicOr(err, eflag);
}

// Volume integral, surface lifting, sources and the Runge-Kutta update of volume_group (separate
// face schedule: the face fluxes 2 F* are read from Fstar), line per thread; UtrNext (optional):
// the traces of the new state (LSRK) or of the state (RHS).
template <int G>
__global__ void __launch_bounds__(G * 16)
    k_volume_line(const NskParams p, float* __restrict__ U, const float* __restrict__ Q,
                  const float* __restrict__ Fstar, float* __restrict__ K, float* __restrict__ Rout, const int mode,
                  const float A, const float B, const double* __restrict__ dtp, const float dtv,
                  int* __restrict__ err, float* __restrict__ UtrNext) {
  using R = float;
  using namespace line;
  extern __shared__ __align__(16) unsigned char line_smem_raw[];
  R* sm = reinterpret_cast<R*>(line_smem_raw);
  const int le = threadIdx.x >> 4, t = threadIdx.x & 15, j = t & 3, kk = t >> 2;
  R* sfs = sm + le * kVolElem;        // [slot][v][fn] 2 F* of the element's faces
  R* sfy = sfs + NF * NV * NFN;       // [v][node] F_y, then the new state
  R* sfz = sfy + NV * NPE;            // [v][node] F_z
  R* tb = sm + G * kVolElem;
  const auto& T = TabSel<R>::get(p);
  const R dt = dtp ? (R)*dtp : dtv;
  const int e = (int)blockIdx.x * G + le;
  const bool valid = e < p.E;
  const size_t nn = (size_t)p.nne, pl = (size_t)NF * p.nfe;
  const int g0 = e * NPE + 4 * t;

  if (valid) {  // face fluxes: Fstar[v][k][E][nfn] holds face (e, +k); slot 2k is the -k neighbour's
    const ElemIdx ex = elem_idx<3>(p, e);
#pragma unroll
    for (int r = 0; r < (NF * NV * 4 + 15) / 16; ++r) {
      const int it = t + 16 * r;
      if (it >= NF * NV * 4) break;
      const int piece = it & 3, v = (it >> 2) % NV, slot = it / (NV * 4), k = slot >> 1;
      const int src = (slot & 1) ? e : nbr_of(p, ex, k, -1);
      stage_copy<true, 4>(sfs + (slot * NV + v) * NFN + 4 * piece,
                          Fstar + (size_t)(v * 3 + k) * p.nfe + (src * NFN + 4 * piece));
    }
  }
  cp_async_commit();
  volume_tables<R, 3, 4>(T, tb, mode == NSK_MODE_RHS ? R(1) : dt);
  R u[NV][4], kin[NV][4], gc[3][4], fx[NV][4];
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float4 a = *reinterpret_cast<const float4*>(U + v * nn + g0);
      u[v][0] = a.x, u[v][1] = a.y, u[v][2] = a.z, u[v][3] = a.w;
    }
    if (mode != NSK_MODE_RHS) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float4 a = *reinterpret_cast<const float4*>(K + v * nn + g0);
        kin[v][0] = a.x, kin[v][1] = a.y, kin[v][2] = a.z, kin[v][3] = a.w;
      }
    }
    float4 qv[NVF];
#pragma unroll
    for (int c = 0; c < NVF; ++c) qv[c] = *reinterpret_cast<const float4*>(Q + c * nn + g0);
    R fy[NV][4], fz[NV][4];
    const R mu = T.mu;
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // volume_node_fluxes
      R tau[3][3];
      int c = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = k; a < 3; ++a) {
          tau[k][a] = f4_at(qv[c++], i);
          tau[a][k] = tau[k][a];
        }
#pragma unroll
      for (int k = 0; k < 3; ++k) gc[k][i] = f4_at(qv[c++], i);
      const R inv = R(1) / u[0][i];
      const R pa = Eos<R>::pa(p, u[0][i]);
      // the symmetric convective momentum flux, each pair k < a once (as volume_node_fluxes)
      R vel[3], off[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) vel[a] = u[1 + a][i] * inv;
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int r = q + 1; r < 3; ++r) off[q][r] = u[1 + q][i] * vel[r];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        R f[NV];
        f[0] = u[1 + k][i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const R fc = (a == k) ? fmaf(u[1 + k][i], vel[k], pa) : (k < a ? off[k][a] : off[a][k]);
          f[1 + a] = fmaf(-mu, tau[k][a], fc);
        }
        f[4] = gc[k][i];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (k == 0) fx[v][i] = f[v];
          if (k == 1) fy[v][i] = f[v];
          if (k == 2) fz[v][i] = f[v];
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      *reinterpret_cast<float4*>(sfy + v * NPE + 4 * t) = f4_make(fy[v]);
      *reinterpret_cast<float4*>(sfz + v * NPE + 4 * t) = f4_make(fz[v]);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  if (valid) {  // volume_residual_update: per node, directions in ascending order
    R res[NV][4], volc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      volc[i] = 0;
#pragma unroll
      for (int v = 0; v < NV; ++v) res[v][i] = 0;
    }
    // the surface and volume terms of direction k for node i, variable v, from the line values fl
    auto term = [&](int v, int i, const R (&dk)[4], const R (&fl)[4], R fp, R fm, R lpk, R lmk) {
      R acc = v == NV - 1 ? volc[i] : res[v][i];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) acc = fmaf(dk[jj], fl[jj], acc);
      if (v == NV - 1) {
        volc[i] = acc;
        res[v][i] = fmaf(fm, lmk, fmaf(-fp, lpk, res[v][i]));
      } else {
        res[v][i] = fmaf(fm, lmk, fmaf(-fp, lpk, acc));
      }
    };
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // x: the thread's own line, face node t
      R dk[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) dk[jj] = tb[i * 4 + jj];
      const R lpk = tb[48 + i], lmk = tb[60 + i];
#pragma unroll
      for (int v = 0; v < NV; ++v)
        term(v, i, dk, fx[v], sfs[(1 * NV + v) * NFN + t], sfs[(0 * NV + v) * NFN + t], lpk, lmk);
    }
    {  // y: lines (jj, kk), face nodes i + 4 kk
      R dk[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) dk[jj] = tb[(4 + j) * 4 + jj];
      const R lpk = tb[48 + 4 + j], lmk = tb[60 + 4 + j];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float4 ln[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) ln[jj] = *reinterpret_cast<const float4*>(sfy + v * NPE + 4 * (jj + 4 * kk));
        const float4 fp = *reinterpret_cast<const float4*>(sfs + (3 * NV + v) * NFN + 4 * kk);
        const float4 fm = *reinterpret_cast<const float4*>(sfs + (2 * NV + v) * NFN + 4 * kk);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const R fl[4] = {f4_at(ln[0], i), f4_at(ln[1], i), f4_at(ln[2], i), f4_at(ln[3], i)};
          term(v, i, dk, fl, f4_at(fp, i), f4_at(fm, i), lpk, lmk);
        }
      }
    }
    {  // z: lines (j, ll), face nodes i + 4 j
      R dk[4];
#pragma unroll
      for (int ll = 0; ll < 4; ++ll) dk[ll] = tb[(8 + kk) * 4 + ll];
      const R lpk = tb[48 + 8 + kk], lmk = tb[60 + 8 + kk];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float4 ln[4];
#pragma unroll
        for (int ll = 0; ll < 4; ++ll) ln[ll] = *reinterpret_cast<const float4*>(sfz + v * NPE + 4 * (j + 4 * ll));
        const float4 fp = *reinterpret_cast<const float4*>(sfs + (5 * NV + v) * NFN + 4 * j);
        const float4 fm = *reinterpret_cast<const float4*>(sfs + (4 * NV + v) * NFN + 4 * j);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const R fl[4] = {f4_at(ln[0], i), f4_at(ln[1], i), f4_at(ln[2], i), f4_at(ln[3], i)};
          term(v, i, dk, fl, f4_at(fp, i), f4_at(fm, i), lpk, lmk);
        }
      }
    }
    const R alpha = tb[tab_smem<3, 4>()], ab = tb[tab_smem<3, 4>() + 1];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      res[NV - 1][i] = fmaf(-T.kb, volc[i], res[NV - 1][i]);
#pragma unroll
      for (int a = 0; a < 3; ++a) res[1 + a][i] = fmaf(alpha * u[0][i], gc[a][i], res[1 + a][i]);
      res[4][i] = fmaf(ab, u[0][i] - u[4][i], res[4][i]);
    }
    if (mode == NSK_MODE_RHS) {
#pragma unroll
      for (int v = 0; v < NV; ++v) *reinterpret_cast<float4*>(Rout + v * nn + g0) = f4_make(res[v]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        R kv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          kv[i] = fmaf(A, kin[v][i], res[v][i]);  // res holds dt R
          u[v][i] = fmaf(B, kv[i], u[v][i]);
        }
        *reinterpret_cast<float4*>(K + v * nn + g0) = f4_make(kv);
        *reinterpret_cast<float4*>(U + v * nn + g0) = f4_make(u[v]);
      }
    }
  }
  if (UtrNext != nullptr) {  // uniform over the grid: the traces of the element's (new) state
    __syncthreads();         // sfy is reused for the state
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; ++v) *reinterpret_cast<float4*>(sfy + v * NPE + 4 * t) = f4_make(u[v]);
#pragma unroll
      for (int s = 0; s < 2; ++s) {  // x faces at face node t, from the thread's own line
        const R* L = s ? T.lp : T.lm;
        R* o = UtrNext + (size_t)s * p.nfe + (e * NFN + t);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          R acc = 0;
#pragma unroll
          for (int i = 0; i < 4; ++i) acc = fmaf(L[i], u[v][i], acc);
          o[v * pl] = acc;
        }
      }
    }
    __syncthreads();
    if (valid) {  // y and z faces: four face nodes of one slot per thread
      const int slot = 2 + (t >> 2), k = slot >> 1, g = t & 3;
      const R* L = (slot & 1) ? T.lp : T.lm;
      R* o = UtrNext + (size_t)slot * p.nfe + (e * NFN + 4 * g);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        R acc[4] = {0, 0, 0, 0};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const float4 ln =
              *reinterpret_cast<const float4*>(sfy + v * NPE + 4 * (k == 1 ? jj + 4 * g : g + 4 * jj));
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i] = fmaf(L[jj], f4_at(ln, i), acc[i]);
        }
        *reinterpret_cast<float4*>(o + v * pl) = f4_make(acc);
      }
    }
  }
}

// One stage of the line schedule: prolongation (when the traces are not ready), line lifting,
// the face pass, line volume + update; a lifting-only stage (mode LIFT, gradients stored) takes
// the node-per-thread lifting. Returns the number of launches or NSK_ERR_CUDA.
template <int G>
int launch_stage_line(const NskParams& p, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  constexpr int smem_lift = (int)sizeof(float) * lift_line_smem<G>();
  constexpr int smem_vol = (int)sizeof(float) * volume_line_smem<G>();
  static const bool attr_ok =
      cudaFuncSetAttribute(k_lift_line<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_lift) == cudaSuccess &&
      cudaFuncSetAttribute(k_volume_line<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_vol) == cudaSuccess;
  if (!attr_ok) return NSK_ERR_CUDA;
  int nl = 0;
  if (l.ev) cudaEventRecord(l.ev[0], s);
  if (!l.traces_ready) {
    k_prolong<float, 3, 4><<<dim3(grid_for(p.nfe, 256), 6), 256, 0, s>>>(p, (const float*)b.U, (float*)b.Utr);
    ++nl;
  }
  if (l.ev) cudaEventRecord(l.ev[1], s);
  const unsigned eb = (unsigned)((p.E + G - 1) / G);
  if (l.mode == NSK_MODE_LIFT) {
    constexpr int GN = group_for<3, 4>(256);
    k_lift<float, 3, 4, GN, false><<<(unsigned)((p.E + GN - 1) / GN), GN * 64, 0, s>>>(
        p, (const float*)b.U, (const float*)b.Utr, (float*)b.Q, (float*)b.FVtr, b.err);
  } else {
    k_lift_line<G><<<eb, G * 16, smem_lift, s>>>(p, (const float*)b.U, (const float*)b.Utr, (float*)b.Q,
                                                 (float*)b.FVtr, b.err);
  }
  if (l.ev) cudaEventRecord(l.ev[2], s);
  ++nl;
  if (l.mode != NSK_MODE_LIFT) {
    k_face<float, 3, 4><<<dim3(grid_for(p.nfe, 256), 3), 256, 0, s>>>(p, (const float*)b.Utr, (const float*)b.FVtr,
                                                                       (float*)b.Fstar, b.err);
    ++nl;
    if (l.ev) cudaEventRecord(l.ev[3], s);
    k_volume_line<G><<<eb, G * 16, smem_vol, s>>>(p, (float*)b.U, (const float*)b.Q, (const float*)b.Fstar,
                                                  (float*)b.K, (float*)l.Rout, l.mode, (float)l.A, (float)l.B,
                                                  l.dt_dev, (float)l.dt_val, b.err, (float*)l.utr_next);
    if (l.ev) cudaEventRecord(l.ev[4], s);
    ++nl;
  }
  if (cudaGetLastError() != cudaSuccess) return NSK_ERR_CUDA;
  return nl;
}

}  // namespace nsk
