// mhd_riemann_vjp.cuh -- reverse-mode derivative of the face solve (riemann<RS> in mhd_device.cuh)
// for the adjoint of the step.
//
// For weights (lf, lap, lam, lus) the scalar g = sum_v lf[v] F[v] + lap alpha+ + lam alpha- +
// lus u* of one face is differentiated with respect to the 15 inputs (left and right face states
// and the normal field) in one reverse sweep. The forward values are recomputed with the same
// device functions (phys_speed, phys_flux, star_state) in double precision, so every branch --
// the max/min of the wave speeds, the HLLD fan region, the degenerate star state, the clamped
// discriminant -- is the one the forward step took, and the derivative is the one of that branch
// (ties and zero square roots as in the forward-mode dual numbers). Each reverse statement is
// the transpose of one forward statement, in reverse order.
#pragma once
#include "mhd_device.cuh"

namespace mhd {

// adjoint of phys_speed (b2, pt, cf2 of a state): accumulates into ds and dbn
__device__ __forceinline__ void phys_speed_rev(const FaceState& s, double bn, double gam, double db2, double dpt,
                                               double dcf2, FaceState& ds, double& dbn) {
  const double bn2 = bn * bn;
  const double b2 = fma(s.by, s.by, fma(s.bz, s.bz, bn2));
  const double P = gam * s.p;
  const double Sp = P + b2;
  const double disc0 = fma(Sp, Sp, (-4.0 * bn2) * P);
  const bool keep = dbits(disc0) >= dbits(0.0);  // pmax(disc, 0) keeps disc
  const double disc = keep ? disc0 : 0.0;
  const double q1 = rsqrt_(disc);
  const double sd = is_zero(disc) ? 0.0 : disc * q1;
  const double r = rcp(s.rho);
  // cf2 = (r / 2) (Sp + sd)
  const double dh = dcf2 * (Sp + sd);
  double dSp = dcf2 * 0.5 * r;
  const double dsd = dSp;
  ds.rho -= 0.5 * dh * r * r;
  // sd = sqrt(disc): derivative rsqrt / 2, taken as 0 at 0
  const double ddisc = (keep && !is_zero(disc)) ? 0.5 * q1 * dsd : 0.0;
  // disc = Sp^2 - 4 bn2 P
  dSp += 2.0 * Sp * ddisc;
  double dbn2 = -4.0 * P * ddisc;
  const double dP = -4.0 * bn2 * ddisc + dSp;  // Sp = P + b2
  double db2t = db2 + dSp;
  ds.p += gam * dP;
  ds.p += dpt;
  db2t += 0.5 * dpt;
  ds.by += 2.0 * s.by * db2t;
  ds.bz += 2.0 * s.bz * db2t;
  dbn2 += db2t;
  dbn += 2.0 * bn * dbn2;
}

// adjoint of phys_flux (U, F, e of a state, given its b2 and pt): dU, dF, de in; accumulates
// into ds, dbn, db2, dpt
__device__ __forceinline__ void phys_flux_rev(const FaceState& s, double bn, double gm1inv, const PhysFlux& o,
                                              const double* dU, const double* dF, double de_extra, FaceState& ds,
                                              double& dbn, double& db2, double& dpt) {
  const double u2 = fma(s.u, s.u, fma(s.v, s.v, s.w * s.w));
  const double ub = fma(s.u, bn, fma(s.v, s.by, s.w * s.bz));
  const double mu = s.rho * s.u;
  const double e = o.e;
  double dmu = dU[1] + dF[0] + dF[1] * s.u + dF[2] * s.v + dF[3] * s.w;
  ds.rho += dU[0] + dU[2] * s.v + dU[3] * s.w;
  ds.v += dU[2] * s.rho + dF[2] * mu;
  ds.w += dU[3] * s.rho + dF[3] * mu;
  const double de = dU[4] + dF[4] * s.u + de_extra;
  ds.u += dF[1] * mu + dF[4] * (e + o.pt);
  dpt += dF[1] + dF[4] * s.u;
  double dbn2 = -dF[1];
  dbn += -dF[2] * s.by - dF[3] * s.bz - dF[4] * ub;
  ds.by -= dF[2] * bn;
  ds.bz -= dF[3] * bn;
  const double dub = -dF[4] * bn;
  ds.u += dub * bn;
  dbn += dub * s.u;
  ds.v += dub * s.by;
  ds.by += dub * s.v;
  ds.w += dub * s.bz;
  ds.bz += dub * s.w;
  ds.p += de * gm1inv;
  ds.rho += de * 0.5 * u2;
  const double du2 = de * 0.5 * s.rho;
  db2 += de * 0.5;
  ds.u += 2.0 * s.u * du2;
  ds.v += 2.0 * s.v * du2;
  ds.w += 2.0 * s.w * du2;
  ds.rho += dmu * s.u;
  ds.u += dmu * s.rho;
  dbn += 2.0 * bn * dbn2;
}

// adjoints of a star state's outputs
struct StarAdj {
  double rs, vs, ws, bys, bzs, es;
};

// adjoint of star_state(q, P, S, SM, ptS, bn, bn2): accumulates into dq, dPe, dPpt, dS, dSM, dptS,
// dbn, dbn2
__device__ __forceinline__ void star_state_rev(const FaceState& q, const PhysFlux& ph, double S, double SM,
                                               double ptS, double bn, double bn2, const StarT<double>& o,
                                               const StarAdj& g, FaceState& dq, double& dPe, double& dPpt,
                                               double& dS, double& dSM, double& dptS, double& dbn, double& dbn2) {
  const double su = S - q.u;
  const double ssm = S - SM;
  const double ssminv = rcp(ssm);
  const double rsu = q.rho * su;
  const double dd = fma(rsu, ssm, -bn2);
  const double scale = fma(rsu, su, bn2);
  const bool degenerate = !vgt(vabs(dd), 1e-12 * scale);
  const double vb = fma(q.u, bn, fma(q.v, q.by, q.w * q.bz));
  const double vbs = fma(SM, bn, fma(o.vs, o.bys, o.ws * o.bzs));
  const double A = fma(su, ph.e, -ph.pt * q.u) + fma(ptS, SM, bn * (vb - vbs));
  double dvs = g.vs, dws = g.ws, dbys = g.bys, dbzs = g.bzs;
  // es = A ssminv
  const double dA = g.es * ssminv;
  double dssminv = g.es * A;
  double dsu = dA * ph.e;
  dPe += dA * su;
  dPpt -= dA * q.u;
  dq.u -= dA * ph.pt;
  dptS += dA * SM;
  dSM += dA * ptS;
  dbn += dA * (vb - vbs);
  const double dvb = dA * bn, dvbs = -dA * bn;
  // vbs = SM bn + vs bys + ws bzs
  dSM += dvbs * bn;
  dbn += dvbs * SM;
  dvs += dvbs * o.bys;
  dbys += dvbs * o.vs;
  dws += dvbs * o.bzs;
  dbzs += dvbs * o.ws;
  // vb = u bn + v by + w bz
  dq.u += dvb * bn;
  dbn += dvb * q.u;
  dq.v += dvb * q.by;
  dq.by += dvb * q.v;
  dq.w += dvb * q.bz;
  dq.bz += dvb * q.w;
  double drsu = 0.0, dssm = 0.0;
  if (degenerate) {
    dq.v += dvs;
    dq.w += dws;
    dq.by += dbys;
    dq.bz += dbzs;
  } else {
    const double ddinv = rcp(dd);
    const double cv = bn * (SM - q.u) * ddinv;
    const double n2 = fma(rsu, su, -bn2);
    const double cb = n2 * ddinv;
    // vs = v - by cv, ws = w - bz cv, bys = by cb, bzs = bz cb
    dq.v += dvs;
    dq.w += dws;
    dq.by += -dvs * cv + dbys * cb;
    dq.bz += -dws * cv + dbzs * cb;
    const double dcv = -dvs * q.by - dws * q.bz;
    const double dcb = dbys * q.by + dbzs * q.bz;
    // cb = n2 ddinv, cv = bn (SM - u) ddinv
    const double dn2 = dcb * ddinv;
    double dddinv = dcb * n2 + dcv * bn * (SM - q.u);
    dbn += dcv * (SM - q.u) * ddinv;
    dSM += dcv * bn * ddinv;
    dq.u -= dcv * bn * ddinv;
    // n2 = rsu su - bn2
    drsu += dn2 * su;
    dsu += dn2 * rsu;
    dbn2 -= dn2;
    // ddinv = 1/dd, dd = rsu ssm - bn2
    const double ddd = -dddinv * ddinv * ddinv;
    drsu += ddd * ssm;
    dssm += ddd * rsu;
    dbn2 -= ddd;
  }
  // rs = rsu ssminv
  drsu += g.rs * ssminv;
  dssminv += g.rs * rsu;
  dssm -= dssminv * ssminv * ssminv;
  // rsu = rho su, ssm = S - SM, su = S - u
  dq.rho += drsu * su;
  dsu += drsu * q.rho;
  dS += dssm + dsu;
  dSM -= dssm;
  dq.u -= dsu;
}

__device__ __forceinline__ void add_side(bool left, FaceState& dl, FaceState& dr, const FaceState& d) {
  FaceState& t = left ? dl : dr;
  t.rho += d.rho;
  t.u += d.u;
  t.v += d.v;
  t.w += d.w;
  t.p += d.p;
  t.by += d.by;
  t.bz += d.bz;
}

// Reverse sweep of hlld(): dF in; accumulates into dsl, dsr, dbn, the adjoints of the two sides'
// b2 / pt (dLb2, dLpt, dRb2, dRpt) and of SL, SR. As in hlld, the side is chosen first, so that
// the one physical flux vector and its reverse are formed by every lane together (outside the fan
// the flux is that vector; inside it the star states' reverse comes first).
__device__ __forceinline__ void hlld_rev(const FaceState& sl, const FaceState& sr, double bn, double gm1inv,
                                         const PhysFlux& Lsp, const PhysFlux& Rsp, double SL, double SR,
                                         const double* dF, FaceState& dsl, FaceState& dsr, double& dbn,
                                         double& dLb2, double& dLpt, double& dRb2, double& dRpt, double& dSL,
                                         double& dSR) {
  // ---- forward values (as in hlld) ----
  const bool supL = gt0(SL);
  const bool fan = !supL && !lt0(SR);
  double sluL = 0.0, sruR = 0.0, mL = 0.0, mR = 0.0, dinv = 0.0, nSM = 0.0, SM = 0.0, nPT = 0.0, ptS = 0.0;
  if (fan) {
    sluL = SL - sl.u;
    sruR = SR - sr.u;
    mL = sluL * sl.rho;
    mR = sruR * sr.rho;
    dinv = rcp(mR - mL);
    nSM = (mR * sr.u - mL * sl.u) + (Lsp.pt - Rsp.pt);
    SM = nSM * dinv;
    nPT = mR * Lsp.pt - mL * Rsp.pt + mL * mR * (sr.u - sl.u);
    ptS = nPT * dinv;
  }
  const bool left = fan ? ge0(SM) : supL;
  const FaceState q = pick(left, sl, sr);
  PhysFlux P;
  P.b2 = left ? Lsp.b2 : Rsp.b2;
  P.pt = left ? Lsp.pt : Rsp.pt;
  phys_flux(q, bn, gm1inv, P);
  // the adjoints of the flux vector's inputs: outside the fan F = P.F
  double dFs[5], dPU[5];
  for (int v = 0; v < 5; ++v) {
    dFs[v] = dF[v];
    dPU[v] = 0.0;
  }
  FaceState dq = {0, 0, 0, 0, 0, 0, 0};
  double dPe = 0.0, dPpt = 0.0, dSM = 0.0, dptS = 0.0, dbn2 = 0.0, dS = 0.0;
  if (fan) {
    const double bn2 = bn * bn;
    const double abn = vabs(bn);
    const double S = left ? SL : SR;
    StarT<double> a;
    star_state(q, P, S, SM, ptS, bn, bn2, a);
    const double isqa = rsqrt_(a.rs);
    const double Ss = left ? SM - abn * isqa : SM + abn * isqa;
    const double Usa[5] = {a.rs, a.rs * SM, a.rs * a.vs, a.rs * a.ws, a.es};
    const bool dstar = hlld_in_rotational(left, SM, a.rs, bn2);

    // ---- reverse ----
    double dUsa[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double dSs = 0.0, disqa = 0.0;
    StarAdj da = {0, 0, 0, 0, 0, 0};
    if (dstar) {
      const FaceState qo = pick(!left, sl, sr);
      const double So = left ? SR : SL;
      StarT<double> b;
      star_state<double, false>(qo, P, So, SM, ptS, bn, bn2, b);
      const double isqb = rsqrt_(b.rs);
      const StarT<double>& sL = left ? a : b;
      const StarT<double>& sR = left ? b : a;
      const double iL = left ? isqa : isqb, iR = left ? isqb : isqa;
      const double sqL = sL.rs * iL, sqR = sR.rs * iR;
      const double sb = sgnd(bn);
      const double inv = rcp(sqL + sqR);
      const double nv = fma(sqL, sL.vs, fma(sqR, sR.vs, (sR.bys - sL.bys) * sb));
      const double nw = fma(sqL, sL.ws, fma(sqR, sR.ws, (sR.bzs - sL.bzs) * sb));
      const double sLR = sqL * sqR;
      const double nby = fma(sqL, sR.bys, fma(sqR, sL.bys, sLR * (sR.vs - sL.vs) * sb));
      const double nbz = fma(sqL, sR.bzs, fma(sqR, sL.bzs, sLR * (sR.ws - sL.ws) * sb));
      const double vss = nv * inv, wss = nw * inv, byss = nby * inv, bzss = nbz * inv;
      const double vbss = fma(SM, bn, fma(vss, byss, wss * bzss));
      const double sq = left ? sqL : sqR;
      const double sgn_side = left ? -1.0 : 1.0;
      const double vbs = fma(SM, bn, fma(a.vs, a.bys, a.ws * a.bzs));
      double Uss[5];
      Uss[0] = a.rs;
      Uss[1] = a.rs * SM;
      Uss[2] = a.rs * vss;
      Uss[3] = a.rs * wss;
      Uss[4] = fma(sgn_side * sq, (vbs - vbss) * sb, a.es);
      // F = Ss (Uss - Usa) + Fs
      double dUss[5];
      for (int v = 0; v < 5; ++v) {
        dSs += dF[v] * (Uss[v] - Usa[v]);
        dUss[v] = Ss * dF[v];
        dUsa[v] -= Ss * dF[v];
      }
      // Uss
      da.rs += dUss[0] + dUss[1] * SM + dUss[2] * vss + dUss[3] * wss;
      dSM += dUss[1] * a.rs;
      double dvss = dUss[2] * a.rs, dwss = dUss[3] * a.rs;
      da.es += dUss[4];
      const double dsq = dUss[4] * sgn_side * (vbs - vbss) * sb;
      const double dvbs = dUss[4] * sgn_side * sq * sb, dvbss = -dvbs;
      // vbs = SM bn + a.vs a.bys + a.ws a.bzs
      dSM += dvbs * bn;
      dbn += dvbs * SM;
      da.vs += dvbs * a.bys;
      da.bys += dvbs * a.vs;
      da.ws += dvbs * a.bzs;
      da.bzs += dvbs * a.ws;
      // vbss = SM bn + vss byss + wss bzss
      dSM += dvbss * bn;
      dbn += dvbss * SM;
      dvss += dvbss * byss;
      const double dbyss = dvbss * vss;
      dwss += dvbss * bzss;
      const double dbzss = dvbss * wss;
      // the four double-star values: X = nX inv
      const double dnv = dvss * inv, dnw = dwss * inv, dnby = dbyss * inv, dnbz = dbzss * inv;
      const double dinv2 = dvss * nv + dwss * nw + dbyss * nby + dbzss * nbz;
      StarAdj dL = {0, 0, 0, 0, 0, 0}, dR = {0, 0, 0, 0, 0, 0};
      double dsqL = 0.0, dsqR = 0.0, dsLR = 0.0;
      if (left) dsqL += dsq; else dsqR += dsq;
      // nv = sqL vsL + sqR vsR + (bysR - bysL) sb
      dsqL += dnv * sL.vs;
      dL.vs += dnv * sqL;
      dsqR += dnv * sR.vs;
      dR.vs += dnv * sqR;
      dR.bys += dnv * sb;
      dL.bys -= dnv * sb;
      // nw
      dsqL += dnw * sL.ws;
      dL.ws += dnw * sqL;
      dsqR += dnw * sR.ws;
      dR.ws += dnw * sqR;
      dR.bzs += dnw * sb;
      dL.bzs -= dnw * sb;
      // nby = sqL bysR + sqR bysL + sLR (vsR - vsL) sb
      dsqL += dnby * sR.bys;
      dR.bys += dnby * sqL;
      dsqR += dnby * sL.bys;
      dL.bys += dnby * sqR;
      dsLR += dnby * (sR.vs - sL.vs) * sb;
      dR.vs += dnby * sLR * sb;
      dL.vs -= dnby * sLR * sb;
      // nbz
      dsqL += dnbz * sR.bzs;
      dR.bzs += dnbz * sqL;
      dsqR += dnbz * sL.bzs;
      dL.bzs += dnbz * sqR;
      dsLR += dnbz * (sR.ws - sL.ws) * sb;
      dR.ws += dnbz * sLR * sb;
      dL.ws -= dnbz * sLR * sb;
      // sLR = sqL sqR; inv = 1/(sqL + sqR)
      dsqL += dsLR * sqR;
      dsqR += dsLR * sqL;
      const double dsum = -dinv2 * inv * inv;
      dsqL += dsum;
      dsqR += dsum;
      // sq = rs i, i = rsqrt(rs)
      double diL = dsqL * sL.rs, diR = dsqR * sR.rs;
      dL.rs += dsqL * iL;
      dR.rs += dsqR * iR;
      // back to sides a (this side) and b (the other)
      StarAdj& dA_ = left ? dL : dR;
      StarAdj& dB_ = left ? dR : dL;
      const double diA = left ? diL : diR, diB = left ? diR : diL;
      da.rs += dA_.rs;
      da.vs += dA_.vs;
      da.ws += dA_.ws;
      da.bys += dA_.bys;
      da.bzs += dA_.bzs;
      disqa += diA;
      StarAdj db = dB_;
      db.es = 0.0;
      db.rs += diB * (-0.5 * isqb * isqb * isqb);
      // b = star_state(qo, ., So, SM, ptS, bn, bn2) without its energy (db.es = 0, so neither the
      // side's flux vectors nor its pt enter)
      FaceState dqo = {0, 0, 0, 0, 0, 0, 0};
      double dPoe = 0.0, dPopt = 0.0, dSo = 0.0;
      star_state_rev(qo, P, So, SM, ptS, bn, bn2, b, db, dqo, dPoe, dPopt, dSo, dSM, dptS, dbn, dbn2);
      add_side(!left, dsl, dsr, dqo);
      if (left) dSR += dSo; else dSL += dSo;
    }
    // Ss = SM -/+ |bn| isqa
    dSM += dSs;
    if (left) { dbn -= dSs * isqa * sgnd(bn); disqa -= dSs * abn; }
    else { dbn += dSs * isqa * sgnd(bn); disqa += dSs * abn; }
    // Fs = S (Usa - P.U) + P.F
    for (int v = 0; v < 5; ++v) {
      dS += dFs[v] * (Usa[v] - P.U[v]);
      dUsa[v] += S * dFs[v];
      dPU[v] = -S * dFs[v];
    }
    // Usa = (rs, rs SM, rs vs, rs ws, es)
    da.rs += dUsa[0] + dUsa[1] * SM + dUsa[2] * a.vs + dUsa[3] * a.ws;
    dSM += dUsa[1] * a.rs;
    da.vs += dUsa[2] * a.rs;
    da.ws += dUsa[3] * a.rs;
    da.es += dUsa[4];
    // isqa = rsqrt(a.rs)
    da.rs += disqa * (-0.5 * isqa * isqa * isqa);
    star_state_rev(q, P, S, SM, ptS, bn, bn2, a, da, dq, dPe, dPpt, dS, dSM, dptS, dbn, dbn2);
  }
  double db2 = 0.0, dpt = dPpt;
  phys_flux_rev(q, bn, gm1inv, P, dPU, dFs, dPe, dq, dbn, db2, dpt);
  add_side(left, dsl, dsr, dq);
  if (left) { dLb2 += db2; dLpt += dpt; } else { dRb2 += db2; dRpt += dpt; }
  if (!fan) return;
  if (left) dSL += dS; else dSR += dS;
  dbn += 2.0 * bn * dbn2;
  // SM = nSM dinv, ptS = nPT dinv, dinv = 1/(mR - mL)
  const double dnSM = dSM * dinv, dnPT = dptS * dinv;
  const double ddinv = dSM * nSM + dptS * nPT;
  const double duRL = sr.u - sl.u;
  double dmR = dnSM * sr.u + dnPT * Lsp.pt + dnPT * mL * duRL;
  double dmL = -dnSM * sl.u - dnPT * Rsp.pt + dnPT * mR * duRL;
  dsr.u += dnSM * mR + dnPT * mL * mR;
  dsl.u -= dnSM * mL + dnPT * mL * mR;
  dLpt += dnSM + dnPT * mR;
  dRpt -= dnSM + dnPT * mL;
  const double dD = -ddinv * dinv * dinv;
  dmR += dD;
  dmL -= dD;
  // mL = (SL - uL) rhoL, mR = (SR - uR) rhoR
  dSL += dmL * sl.rho;
  dsl.u -= dmL * sl.rho;
  dsl.rho += dmL * sluL;
  dSR += dmR * sr.rho;
  dsr.u -= dmR * sr.rho;
  dsr.rho += dmR * sruR;
}

// Gradient of g = sum_v lf[v] F[v] + lap ap + lam am + lus u* of riemann<RS>(sl, sr, bn) in
// (sl, sr, bn), written into dsl, dsr, dbn.
template <int RS>
__device__ __forceinline__ void riemann_vjp(const FaceState& sl, const FaceState& sr, double bn, double gam,
                                            double gm1inv, const double* lf, double lap, double lam, double lus,
                                            FaceState& dsl, FaceState& dsr, double& dbn) {
  dsl = {0, 0, 0, 0, 0, 0, 0};
  dsr = {0, 0, 0, 0, 0, 0, 0};
  dbn = 0.0;
  // ---- forward (as in riemann) ----
  PhysFlux L, R;
  phys_speed(sl, bn, gam, L);
  phys_speed(sr, bn, gam, R);
  double SL = 0.0, SR = 0.0, ap, am;
  bool llf_left = true, cmax_left = true, umax_left = true, umin_left = true, ap_pos = true, am_pos = true;
  if (RS == RS_LLF) {
    const double aL = vabs(sl.u) + sqrt_(L.cf2), aR = vabs(sr.u) + sqrt_(R.cf2);
    llf_left = dbits(aL) >= dbits(aR);
    ap = am = llf_left ? aL : aR;
  } else {
    cmax_left = dbits(L.cf2) >= dbits(R.cf2);
    const double cmax = sqrt_(cmax_left ? L.cf2 : R.cf2);
    umax_left = okey(sl.u) >= okey(sr.u);
    umin_left = okey(sl.u) <= okey(sr.u);
    const double umax = umax_left ? sl.u : sr.u, umin = umin_left ? sl.u : sr.u;
    SR = umax + cmax;
    SL = umin - cmax;
    ap_pos = !(okey(0.0) >= okey(SR));  // vmax(0, SR) picks SR
    am_pos = !(okey(0.0) >= okey(cmax - umin));
    ap = ap_pos ? SR : 0.0;
    am = am_pos ? cmax - umin : 0.0;
  }
  const double sum = ap + am;
  const bool zero = is_zero(sum);
  const double inv = zero ? 0.0 : rcp(sum);

  // ---- reverse ----
  double dap = lap, dam = lam;
  double dLb2 = 0.0, dLpt = 0.0, dRb2 = 0.0, dRpt = 0.0, dLcf = 0.0, dRcf = 0.0;
  // u* = (ap uL + am uR) inv, or uL when ap + am = 0
  if (zero) {
    dsl.u += lus;
  } else {
    const double n = fma(ap, sl.u, am * sr.u);
    const double dn = lus * inv;
    const double dinv = lus * n;
    dap += dn * sl.u;
    dsl.u += dn * ap;
    dam += dn * sr.u;
    dsr.u += dn * am;
    const double ds = -dinv * inv * inv;
    dap += ds;
    dam += ds;
  }
  double dSL = 0.0, dSR = 0.0;
  if (RS == RS_HLLD) {
    hlld_rev(sl, sr, bn, gm1inv, L, R, SL, SR, lf, dsl, dsr, dbn, dLb2, dLpt, dRb2, dRpt, dSL, dSR);
  } else {
    phys_flux(sl, bn, gm1inv, L);
    phys_flux(sr, bn, gm1inv, R);
    double dUL[5], dFL[5], dUR[5], dFR[5];
    if (zero) {
      for (int v = 0; v < 5; ++v) { dFL[v] = lf[v]; dUL[v] = 0.0; dFR[v] = 0.0; dUR[v] = 0.0; }
    } else {
      // F = wl FL + wr FR - wd (UR - UL), wl = ap inv, wr = am inv, wd = ap am inv
      const double wl = ap * inv, wr = am * inv, wd = ap * am * inv;
      double dwl = 0.0, dwr = 0.0, dwd = 0.0;
      for (int v = 0; v < 5; ++v) {
        dwl += lf[v] * L.F[v];
        dwr += lf[v] * R.F[v];
        dwd -= lf[v] * (R.U[v] - L.U[v]);
        dFL[v] = lf[v] * wl;
        dFR[v] = lf[v] * wr;
        dUR[v] = -lf[v] * wd;
        dUL[v] = lf[v] * wd;
      }
      dap += dwl * inv + dwd * am * inv;
      dam += dwr * inv + dwd * ap * inv;
      const double dinv = dwl * ap + dwr * am + dwd * ap * am;
      const double ds = -dinv * inv * inv;
      dap += ds;
      dam += ds;
    }
    phys_flux_rev(sl, bn, gm1inv, L, dUL, dFL, 0.0, dsl, dbn, dLb2, dLpt);
    phys_flux_rev(sr, bn, gm1inv, R, dUR, dFR, 0.0, dsr, dbn, dRb2, dRpt);
  }
  // wave speeds
  if (RS == RS_LLF) {
    const double da = dap + dam;
    if (llf_left) {
      dsl.u += neg_if(dbits(sl.u) < 0, da);
      dLcf += da;
    } else {
      dsr.u += neg_if(dbits(sr.u) < 0, da);
      dRcf += da;
    }
  } else {
    // ap = max(0, SR), am = max(0, cmax - umin), SR = umax + cmax, SL = umin - cmax
    if (ap_pos) dSR += dap;
    double dcmax = dSR - dSL, dumin = dSL;
    const double dumax = dSR;
    if (am_pos) {
      dcmax += dam;
      dumin -= dam;
    }
    if (cmax_left) dLcf += dcmax; else dRcf += dcmax;
    if (umax_left) dsl.u += dumax; else dsr.u += dumax;
    if (umin_left) dsl.u += dumin; else dsr.u += dumin;
  }
  // cf = sqrt(cf2) (the larger speed is the square root of the larger square): derivative
  // rsqrt / 2, taken as 0 at 0
  const double dLcf2 = is_zero(L.cf2) ? 0.0 : 0.5 * rsqrt_(L.cf2) * dLcf;
  const double dRcf2 = is_zero(R.cf2) ? 0.0 : 0.5 * rsqrt_(R.cf2) * dRcf;
  phys_speed_rev(sl, bn, gam, dLb2, dLpt, dLcf2, dsl, dbn);
  phys_speed_rev(sr, bn, gam, dRb2, dRpt, dRcf2, dsr, dbn);
}

}  // namespace mhd
