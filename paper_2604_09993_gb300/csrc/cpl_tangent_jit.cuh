// cpl_tangent_jit.cuh — device source of the coupled path's tangent kernel,
// compiled at run time (NVRTC) once per model shape.  The library prepends a
// prelude that fixes, as compile-time constants, everything but the robot's
// numbers: the sizes (NB, NJ, NC, NXT, NU, NL, NQD, NK, ...), the joint and
// contact topology, the live / quadrature row maps, the skyline structure of
// K and the stage-data layout.  Every loop over links, joints, contacts and
// rows is then unrolled with static indices, so the column's state (live
// rows, stage values, quadrature rows, generalized-force tangent, KKT
// right-hand side) lives in registers instead of runtime-indexed shared
// memory; RKF45's stored stage slopes stay in shared memory.  The arithmetic
// is that of k_cpl_tangent in coupled.cu (see its comments): per stage, the
// derivative of the right-hand side along the column's stage tangent with one
// solve by the recorded L D L^T factor of K, then the Runge-Kutta update.
//
// The prelude defines: CPL_TP (float or double), CPL_SCH (0 RK4, 1 RKF45),
// CPL_BS (threads per block), the integer constants, the __device__
// constexpr tables JPAR, JCHI, NPOS, NF, NOFF, CBODY, CONTACT, LROW, QROW,
// LINV, QINV, CPERM, and the scheme's tableau TAB_A, TAB_B, TAB_C and
// TAB_BETA (beta_l = sum_j b_j a_jl) as __constant__ arrays in CPL_TP.
constexpr int SCH = CPL_SCH;
constexpr int BS = CPL_BS;
constexpr int NSTG = SCH ? 6 : 4;  // stages
constexpr int NKS = SCH ? 5 : 1;   // stored slopes

struct Num {
  TP minv[NB], iinv[NB];
};

extern "C" __global__ void __launch_bounds__(BS) cpl_tangent(const __grid_constant__ Num P, long i0,
                                                            long n, int nsub,
                                                            const double* __restrict__ s,
                                                            const TP* __restrict__ sd,
                                                            TP* __restrict__ A, TP* __restrict__ Bm,
                                                            TP* __restrict__ Bp, TP* __restrict__ S,
                                                            unsigned* status, int layout,
                                                            const int2* __restrict__ entries,
                                                            const ciscvx::InstRec* __restrict__ inst,
                                                            int cmp) {
  extern __shared__ __align__(16) unsigned char jit_smem[];
  TP* ksh = reinterpret_cast<TP*>(jit_smem) + threadIdx.x;  // stored slopes (RKF45), element major
  const long g = (long)blockIdx.x * BS + threadIdx.x;
  const long t = g / CNT;
  if (t >= n) return;
  const int col = CPERM[g - t * CNT];

  constexpr int NQ = 3 * NB;
  int qin = -1;
  bool right = false, scol = false;
  if (col >= NXT) {
    if (col < NXT + NU) qin = col - NXT;
    else if (col < NXT + 2 * NU) { qin = col - NXT - NU; right = true; }
    else scol = true;
  }
  TP PL[NL], XS[NL], PQ[NQD > 0 ? NQD : 1], ACC[NL], KST[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) PL[l] = (LINV[l] == col) ? TP(1) : TP(0);
#pragma unroll
  for (int q = 0; q < NQD; ++q) PQ[q] = (QINV[q] == col) ? TP(1) : TP(0);
  const long long astride = cmp ? (long long)COLPTR[NXT] : (long long)NXT * NXT;
  const TP sk = TP(s[ciscvx::iv_ref(i0 + t, NXT, NU, NC, layout, entries, inst, astride).s]);
  const TP h = TP(1) / TP(nsub);
  const TP hsk = h * sk;
  const TP* sdk = sd + (size_t)t * nsub * NSTG * SD_SIZE;

  for (int i = 0; i < nsub; ++i) {
    // quadrature rows: p += h s v at the substep start
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (CONTACT[b] >= 0) continue;
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2) PQ[QROW[3 * b + c2]] += hsk * PQ[QROW[NQ + 3 * b + c2]];
    }
    for (int j = 0; j < NSTG; ++j) {
      const TP* D = sdk + (size_t)(i * NSTG + j) * SD_SIZE;
      const TP* F = D + SD_F;
      const TP bj = TAB_B[j], hbj = h * bj, h2b = h * h * sk * TAB_BETA[j];
      // stage tangent of the live rows
#pragma unroll
      for (int l = 0; l < NL; ++l) XS[l] = PL[l];
      if (SCH) {
        for (int m = 0; m < j; ++m) {
          const TP ah = TAB_A(j, m) * h;
          if (ah == TP(0)) continue;
#pragma unroll
          for (int l = 0; l < NL; ++l) XS[l] += ah * ksh[(m * NL + l) * BS];
        }
      } else if (j > 0) {
        const TP ah = TAB_A(j, j - 1) * h;
#pragma unroll
        for (int l = 0; l < NL; ++l) XS[l] += ah * KST[l];
      }
      const TP tau = (TP(i) + TAB_C[j]) * h;
      const TP w = qin < 0 ? TP(0) : (right ? tau : TP(1) - tau);
      // generalized-force tangent e: -dtheta QW (moving application points) + direct inputs
      TP e[3 * NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        e[3 * b] = TP(0);
        e[3 * b + 1] = TP(0);
        e[3 * b + 2] = -XS[LROW[3 * b + 2]] * D[SD_QW + b];
      }
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        if (qin == jj) {
          e[3 * JCHI[jj] + 2] += w;
          e[3 * JPAR[jj] + 2] -= w;
        }
        if (!JELIM) {
#pragma unroll
          for (int cp = 0; cp < 2; ++cp) {
            if (qin != NJ + 2 * jj + cp) continue;
#pragma unroll
            for (int role = 0; role < 2; ++role) {
              const int b = role ? JPAR[jj] : JCHI[jj];
              const TP rx = D[SD_ARM + 4 * jj + 2 * role], ry = D[SD_ARM + 4 * jj + 2 * role + 1];
              const TP sw = role ? -w : w;
              e[3 * b + cp] += sw;
              e[3 * b + 2] += sw * (cp ? rx : -ry);
            }
          }
        }
      }
      // contacts: force tangent and the auxiliary rows
#pragma unroll
      for (int ic = 0; ic < NC; ++ic) {
        const int b = CBODY[ic];
        const TP* Dc = D + SD_CON + NCF * ic;
        const TP rx = Dc[0], ry = Dc[1];
        const TP dth = XS[LROW[3 * b + 2]];
        const TP dxc = XS[LROW[3 * b]] - ry * dth;
        const TP dyc = XS[LROW[3 * b + 1]] + rx * dth;
        TP dft = TP(0), dfn = TP(0), dga = TP(0);
        const int qc = qin - (CI0 + 3 * ic);
        if (AUX) {
          if (qc == 0) dft = w;
          if (qc == 1) dfn = w;
          if (qc == 2) dga = w;
        } else {
          if (qc == 0) dfn = w;
          if (qc == 1) dft = w;
          if (qc == 2) dft = -w;
        }
        const TP dfx = Dc[2] * dft + Dc[4] * dfn + Dc[6] * dxc;
        const TP dfy = Dc[3] * dft + Dc[5] * dfn + Dc[7] * dxc;
        e[3 * b] += dfx;
        e[3 * b + 1] += dfy;
        e[3 * b + 2] += rx * dfy - ry * dfx;
        const TP dphi = Dc[8] * dxc + Dc[9] * dyc;
        if (!AUX) {
          TP dy = Dc[10] * dphi;
          if (qc >= 0 && qc < 3) dy += Dc[11 + qc] * w;
          TP kv = sk * dy;
          if (scol) kv += F[6 * NB + ic];
          PQ[QROW[6 * NB + ic]] += hbj * kv;
        } else {
          // lambda^c = t . v_c + gamma phi_t / sqrt(1 + phi_t^2), v_c = (v_x - omega r_y, v_y + omega r_x)
          const TP om = F[3 * b + 2];
          const TP dom = XS[LROW[NQ + 3 * b + 2]];
          const TP dvcx = XS[LROW[NQ + 3 * b]] - dom * ry - om * rx * dth;
          const TP dvcy = XS[LROW[NQ + 3 * b + 1]] + dom * rx - om * ry * dth;
          const TP dys[5] = {dfn,
                             Dc[16] * dxc + Dc[2] * dvcx + Dc[3] * dvcy + Dc[17] * dft + Dc[18] * dga,
                             dga, Dc[19] * dft + Dc[20] * dfn,
                             Dc[10] * dphi + Dc[11] * dft + Dc[12] * dfn + Dc[13] * dga};
          const int rows[5] = {6 * NB + 4 * ic, 6 * NB + 4 * ic + 1, 6 * NB + 4 * ic + 2,
                               6 * NB + 4 * ic + 3, 6 * NB + 4 * NC + ic};
#pragma unroll
          for (int y = 0; y < 5; ++y) {
            TP kv = sk * dys[y];
            if (scol) kv += F[rows[y]];
            PQ[QROW[rows[y]]] += hbj * kv;
          }
        }
      }
      // Eq. (3): K dlambda = sum over joint ends s (alpha domega + beta dtheta - e_lin / m - perp(r) e_ang / I)
      if (JELIM && NK > 0) {
        TP x[NK > 0 ? NK : 1];
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
          TP a0 = TP(0), a1 = TP(0);
#pragma unroll
          for (int role = 0; role < 2; ++role) {
            const int b = role ? JPAR[jj] : JCHI[jj];
            const TP rx = D[SD_ARM + 4 * jj + 2 * role], ry = D[SD_ARM + 4 * jj + 2 * role + 1];
            const TP om = F[3 * b + 2], omd = F[NQ + 3 * b + 2];
            const TP dth = XS[LROW[3 * b + 2]], dom = XS[LROW[NQ + 3 * b + 2]];
            const TP ea = e[3 * b + 2] * P.iinv[b];
            const TP c0 = TP(2) * om * rx * dom + (-om * om * ry + omd * rx) * dth - e[3 * b] * P.minv[b] + ry * ea;
            const TP c1 = TP(2) * om * ry * dom + (om * om * rx + omd * ry) * dth - e[3 * b + 1] * P.minv[b] - rx * ea;
            if (role) { a0 -= c0; a1 -= c1; } else { a0 += c0; a1 += c1; }
          }
          x[2 * NPOS[jj]] = a0;
          x[2 * NPOS[jj] + 1] = a1;
        }
        const TP* Kf = D + SD_K;
#pragma unroll
        for (int ii = 1; ii < NK; ++ii) {
          TP acc = x[ii];
#pragma unroll
          for (int kk = 0; kk < ii; ++kk)
            if (kk >= NF[ii]) acc -= Kf[NOFF[ii] + kk - NF[ii]] * x[kk];
          x[ii] = acc;
        }
#pragma unroll
        for (int ii = NK - 1; ii >= 0; --ii) {
          TP acc = x[ii] * Kf[NOFF[ii] + ii - NF[ii]];
#pragma unroll
          for (int kk = ii + 1; kk < NK; ++kk)
            if (NF[kk] <= ii) acc -= Kf[NOFF[kk] + ii - NF[kk]] * x[kk];
          x[ii] = acc;
        }
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
          const TP lx = x[2 * NPOS[jj]], ly = x[2 * NPOS[jj] + 1];
#pragma unroll
          for (int role = 0; role < 2; ++role) {
            const int b = role ? JPAR[jj] : JCHI[jj];
            const TP rx = D[SD_ARM + 4 * jj + 2 * role], ry = D[SD_ARM + 4 * jj + 2 * role + 1];
            const TP sx = role ? -lx : lx, sy = role ? -ly : ly;
            e[3 * b] += sx;
            e[3 * b + 1] += sy;
            e[3 * b + 2] += rx * sy - ry * sx;
          }
        }
      }
      // slopes: live rows (stage recursion) and quadrature rows
      auto live = [&](int row, TP dy) {
        TP kv = sk * dy;
        if (scol) kv += F[row];
        const int l = LROW[row];
        if (NKS == 1) {
          if (j < NSTG - 1) KST[l] = kv;
          ACC[l] = (j == 0) ? bj * kv : ACC[l] + bj * kv;
          if (j == NSTG - 1) PL[l] += h * ACC[l];
        } else if (j < NSTG - 1) {
          ksh[(j * NL + l) * BS] = kv;
        } else {  // last stage: x += h sum_m b_m k_m from the stored slopes (b_2 = 0)
          TP acc = bj * kv;
#pragma unroll
          for (int m = NSTG - 2; m >= 0; --m)
            if (m != 1) acc += TAB_B[m] * ksh[(m * NL + l) * BS];
          PL[l] += h * acc;
        }
      };
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const TP dv0 = e[3 * b] * P.minv[b], dv1 = e[3 * b + 1] * P.minv[b];
        const TP dw = e[3 * b + 2] * P.iinv[b];
        live(3 * b + 2, XS[LROW[NQ + 3 * b + 2]]);
        live(NQ + 3 * b + 2, dw);
        if (CONTACT[b] >= 0) {
          live(3 * b, XS[LROW[NQ + 3 * b]]);
          live(3 * b + 1, XS[LROW[NQ + 3 * b + 1]]);
          live(NQ + 3 * b, dv0);
          live(NQ + 3 * b + 1, dv1);
        } else {
          const TP dv[2] = {dv0, dv1};
#pragma unroll
          for (int c2 = 0; c2 < 2; ++c2) {
            TP kv = sk * dv[c2];
            TP pinc = TP(0);
            if (scol) {
              kv += F[NQ + 3 * b + c2];
              pinc = h2b * F[NQ + 3 * b + c2];
              if (j == 0) pinc += h * F[3 * b + c2];
            }
            PQ[QROW[3 * b + c2]] += h2b * kv + pinc;
            PQ[QROW[NQ + 3 * b + c2]] += hbj * kv;
          }
        }
      }
    }
  }
  // column `col` of [A | B- | B+ | S]
  TP* out;
  size_t stride;
  const ciscvx::IvRef ad = ciscvx::iv_ref(i0 + t, NXT, NU, NC, layout, entries, inst, astride);
  if (cmp) {  // compact: column-major, the column's rows contiguous
    if (col < NXT) out = A + ad.a + COLPTR[col];
    else if (!scol) out = (right ? Bp : Bm) + ad.b + (size_t)qin * NXT;
    else out = S + ad.v;
    stride = 1;
  } else if (col < NXT) { out = A + ad.a + col; stride = NXT; }
  else if (!scol) { out = (right ? Bp : Bm) + ad.b + qin; stride = NU; }
  else { out = S + ad.v; stride = 1; }
  float chk = 0.0f;
#pragma unroll
  for (int r = 0; r < NXT; ++r) {
    const TP v = LROW[r] >= 0 ? PL[LROW[r]] : PQ[QROW[r]];
    out[(size_t)r * stride] = v;
    chk += float(v);
  }
  if (!isfinite(chk)) atomicOr(status, 1u);
}
