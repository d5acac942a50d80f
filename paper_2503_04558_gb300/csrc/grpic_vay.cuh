// grpic_vay.cuh -- the alternative momentum update of Sec. 2.2: Vay's
// update (Vay 2008, Phys. Plasmas 15, 056701) in the frame of the normal
// observer (FIDO), written with the 3-metric instead of an explicit triad.
//
// In any orthonormal triad of gamma_ij the Lorentz force of Eq. Lorentz is
// the flat one over the FIDO's proper time alpha dt, with fields D and B, so
// the triad step  u' = u + h (E + (u / Gamma) x B / 2),  h = (q/m) alpha dt,
// tau = h B / 2,  sigma = 1 + u'.u' - tau.tau,
// Gamma1 = sqrt((sigma + sqrt(sigma^2 + 4 (tau.tau + (u'.tau)^2))) / 2),
// t = tau / Gamma1,  s = 1 / (1 + t.t),  u1 = s (u' + (u'.t) t + u' x t)
// maps to coordinate components through dot products gamma^ij u_i w_j (two
// covectors), u_i V^i (covector and vector), gamma_ij V^i W^j (two vectors)
// and cross products e_ijk V^j W^k, e_ijk = sqrt(gamma) eps_ijk, of two
// vectors (a covector is raised first).  The result does not depend on the
// triad (the step uses only dot and cross products).
#pragma once

namespace grpic {

// metric quantities at the particle: lapse, gamma_ij, gamma^ij, sqrt(gamma)
// (the r-phi block plus theta-theta of Kerr-Schild)
template <typename T>
struct VayMetric {
    T alpha, g_rr, g_rp, g_tt, g_pp, gi_rr, gi_rp, gi_tt, gi_pp, sqrtg;
};

template <typename T>
__device__ __forceinline__ void vay_step(const VayMetric<T> &m, T qm, T dt, const T D[3], const T B[3], T u[3])
{
    // E_i = gamma_ij D^j;  v^j = gamma^jl u_l / Gamma
    const T E0 = m.g_rr * D[0] + m.g_rp * D[2], E1 = m.g_tt * D[1], E2 = m.g_rp * D[0] + m.g_pp * D[2];
    const T w0 = m.gi_rr * u[0] + m.gi_rp * u[2], w1 = m.gi_tt * u[1], w2 = m.gi_rp * u[0] + m.gi_pp * u[2];
    const T G = sqrt(T(1) + u[0] * w0 + u[1] * w1 + u[2] * w2);
    const T iG = T(1) / G;
    const T h = qm * m.alpha * dt;
    const T hs = T(0.5) * h * m.sqrtg * iG;
    // u'_i = u_i + h E_i + (h / 2) e_ijk v^j B^k
    const T p0 = u[0] + h * E0 + hs * (w1 * B[2] - w2 * B[1]);
    const T p1 = u[1] + h * E1 + hs * (w2 * B[0] - w0 * B[2]);
    const T p2 = u[2] + h * E2 + hs * (w0 * B[1] - w1 * B[0]);
    // tau^k = h B^k / 2
    const T t0 = T(0.5) * h * B[0], t1 = T(0.5) * h * B[1], t2 = T(0.5) * h * B[2];
    const T tl0 = m.g_rr * t0 + m.g_rp * t2, tl1 = m.g_tt * t1, tl2 = m.g_rp * t0 + m.g_pp * t2;
    const T tt = t0 * tl0 + t1 * tl1 + t2 * tl2;
    const T us = p0 * t0 + p1 * t1 + p2 * t2;
    const T q0 = m.gi_rr * p0 + m.gi_rp * p2, q1 = m.gi_tt * p1, q2 = m.gi_rp * p0 + m.gi_pp * p2;
    const T sigma = T(1) + p0 * q0 + p1 * q1 + p2 * q2 - tt;
    const T G1 = sqrt(T(0.5) * (sigma + sqrt(sigma * sigma + T(4) * (tt + us * us))));
    const T iG1 = T(1) / G1;
    const T s = T(1) / (T(1) + tt * iG1 * iG1);
    // u1_i = s (u'_i + (u'.t) t_i + e_ijk u'^j t^k), t = tau / Gamma1
    const T ut = us * iG1 * iG1;        // (u'.t) with t_i = tl_i / Gamma1
    const T cs = m.sqrtg * iG1;
    u[0] = s * (p0 + ut * tl0 + cs * (q1 * t2 - q2 * t1));
    u[1] = s * (p1 + ut * tl1 + cs * (q2 * t0 - q0 * t2));
    u[2] = s * (p2 + ut * tl2 + cs * (q0 * t1 - q1 * t0));
}

}  // namespace grpic
