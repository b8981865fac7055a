// kmc_mean.cuh -- the Ref. [8] mode on the device (Sec. II.3): the mean
// magnetisation of non-interacting NPs, obtained by carrying the probability of
// each energy well instead of sampling jumps. Included only by kmc_step.cu,
// which owns the grid tables and the Eq. 2 helpers it uses.
//
// With no dipolar field the total field stays along z, so each NP keeps one
// working plane for the whole run: the plane of its easy axis a and z, with
// e_perp the unit vector of z normal to a (or a fallback when a is along z).
// The field enters Eq. 2 at the angle phi_z between a and z, or phi_z + pi
// when the field is negative. At every step, per NP (one thread, FP64):
//   * extrema of Eq. 2 by the 200-node scan and Newton (as in the kMC step);
//   * with one minimum all probability sits in it; with two, the probability
//     of each old well moves to the new minimum whose basin (the arc between
//     the two maxima) contains the old well's angle;
//   * Eqs. 3-5 relax the two-well occupation towards its equilibrium over
//     t_step: p_A <- p_A,inf + (p_A - p_A,inf) e^{-(nu_A + nu_B) t_step},
//     p_A,inf = nu_B / (nu_A + nu_B), the barrier top being the lower maximum;
//   * <m_z> = sum_w p_w (cos th_w a_z + sin th_w e_perp,z), added volume-
//     weighted to the lysosome's loop record in 64-bit fixed point.
#pragma once

namespace kmc {

constexpr int kMeanWarps = 4;

__global__ void __launch_bounds__(kMeanWarps * 32) kmc_mean_kernel(const MeanArgs a) {
  __shared__ GridTables<double> tab;
  tab.load();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * kMeanWarps + warp;
  if (item >= a.n_items) return;  // the whole warp
  const MeanItem it = a.items[item];
  const MeanLysDev L = a.lys[it.l];
  const bool active = lane < it.nt;
  const int i = L.off + it.t0 + min(lane, it.nt - 1);
  const dbl4 ax = a.axis[i];
  const double beta = a.beta[i], vfrac = a.vfrac[i];
  const double pi = 0.5 * Prec<double>::two_pi;
  // the fixed working plane: e_perp = normalise(z - (z.a) a)
  double px = -ax.z * ax.x, py = -ax.z * ax.y, pz = 1.0 - ax.z * ax.z;
  double sp = sqrt(px * px + py * py + pz * pz);
  double phz;
  if (sp >= 1e-12) {
    phz = atan2(sp, ax.z);
  } else {  // a along z: any normal will do
    if (fabs(ax.x) > 0.9) {
      px = -ax.z;
      py = 0.0;
      pz = ax.x;
    } else {
      px = 0.0;
      py = ax.z;
      pz = -ax.y;
    }
    sp = sqrt(px * px + py * py + pz * pz);
    phz = (ax.z >= 0.0) ? 0.0 : pi;
  }
  const double epz = pz / sp;
  // start: all probability in the well along +-a with m_z >= 0
  int nw = 1;
  double thw0 = (ax.z >= 0.0) ? 0.0 : pi, thw1 = 0.0, pw0 = 1.0, pw1 = 0.0;
  Profile<double> pf;
  pf.k = L.k;
  pf.k2 = 2.0 * L.k;
  const double h = tab.th[1] - tab.th[0];
  bool bad = false;
  for (int p = 0; p < a.periods; ++p) {
    for (int k = 0; k < a.S; ++k) {
      const double H = L.bmax * a.cos_k[k];
      const double phi = (H < 0.0) ? phz + pi : phz;
      double sphi, cphi;
      sincos(phi, &sphi, &cphi);
      const double b = fabs(H);
      pf.bc = b * cphi;
      pf.bs = b * sphi;
      // step iv: brackets in grid order, then Newton in each
      int cnt = 0;
      double th[4], en[4];
      bool is_min[4];
      const double d_first = pf.d1(tab.sc[0].x, tab.sc[0].y);
      double left = d_first;
      for (int j = 0; j < kGrid; ++j) {
        const double right = (j + 1 < kGrid) ? pf.d1(tab.sc[j + 1].x, tab.sc[j + 1].y) : d_first;
        if ((left < 0.0) != (right < 0.0)) {
          if (cnt < 4) {
            double s, c;
            const double off = refine_in_cell(pf, tab.sc[j].x, tab.sc[j].y, h, left, right, s, c);
            double t = tab.th[j] + off;
            if (t >= Prec<double>::two_pi) t -= Prec<double>::two_pi;
            th[cnt] = t;
            en[cnt] = pf.e(s, c);
            is_min[cnt] = left < 0.0;
          }
          ++cnt;
        }
        left = right;
      }
      int nmin = 0, nmax = 0, imin0 = 0, imin1 = 0, imax0 = 0, imax1 = 0;
      for (int q = 0; q < min(cnt, 4); ++q) {
        if (is_min[q]) {
          if (nmin == 0) imin0 = q; else if (nmin == 1) imin1 = q;
          ++nmin;
        } else {
          if (nmax == 0) imax0 = q; else if (nmax == 1) imax1 = q;
          ++nmax;
        }
      }
      const bool skip = cnt > 4 || nmin > 2 || nmax > 2;
      bad = bad || (active && skip);
      if (!skip) {
        if (nmin == 1) {
          nw = 1;
          thw0 = th[imin0];
          pw0 = 1.0;
        } else if (nmin == 2) {
          const double M1 = th[imax0], M2 = th[imax1];
          const bool arcA = on_arc<double>(th[imin0], M1, M2);
          double pn0 = 0.0, pn1 = 0.0;
          if (on_arc<double>(thw0, M1, M2) == arcA) pn0 += pw0; else pn1 += pw0;
          if (nw == 2) {
            if (on_arc<double>(thw1, M1, M2) == arcA) pn0 += pw1; else pn1 += pw1;
          }
          if (!L.t_zero) {
            // Eqs. 3-5 with nu t_step = exp(ln(t_step / tau0) - beta dE)
            const double e3 = fmin(en[imax0], en[imax1]);
            const double nuA = exp(L.lognu0t - beta * (e3 - en[imin0]));
            const double nuB = exp(L.lognu0t - beta * (e3 - en[imin1]));
            const double sum = nuA + nuB;
            if (sum > 0.0) {
              const double decay = exp(-sum);
              const double pinf = nuB / sum;
              const double pA = pinf + (pn0 - pinf) * decay;
              pn1 = 1.0 - pA;
              pn0 = pA;
            }
          }
          nw = 2;
          thw0 = th[imin0];
          thw1 = th[imin1];
          pw0 = pn0;
          pw1 = pn1;
        }
      }
      if (p >= a.discard) {
        double mz = pw0 * (cos(thw0) * ax.z + sin(thw0) * epz);
        if (nw == 2) mz += pw1 * (cos(thw1) * ax.z + sin(thw1) * epz);
        double c = (active && !skip) ? vfrac * mz : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) {
          const long long rec = static_cast<long long>(p - a.discard) * a.S + k;
          atomicAdd(reinterpret_cast<unsigned long long *>(
                        &a.loop[static_cast<long long>(it.l) * a.n_rec + rec]),
                    static_cast<unsigned long long>(__double2ll_rn(c * kLoopScale)));
        }
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, kErrExtrema);
}

}  // namespace kmc
