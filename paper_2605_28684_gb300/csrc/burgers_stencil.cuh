// FP64 Burgers stencil of the gradient pass: f_i, its Jacobian row and its
// viscosity derivative (Sec. 5.1 problem setup).
//
// f_i = -(F_{i+1/2} - F_{i-1/2}) N + nu (u_{i+1} - 2 u_i + u_{i-1}) N^2 with the
// Godunov flux F(uL, uR) = max(max(uL,0)^2/2, min(uR,0)^2/2); the Jacobian row
// (dl, dc, dr) = (df_i/du_{i-1}, df_i/du_i, df_i/du_{i+1}) takes the
// derivative of the selected branch (tie -> left); df_i/dnu is the centred
// second difference times N^2.
#pragma once

namespace rom {

struct StencilRow {
  double f, dl, dc, dr, fnu;
};

__device__ __forceinline__ StencilRow burgers_stencil(double ul, double u, double ur, double nu,
                                                      double inv_dx) {
  const double Ll = 0.5 * fmax(ul, 0.0) * fmax(ul, 0.0);
  const double Rl = 0.5 * fmin(u, 0.0) * fmin(u, 0.0);
  const bool tl = Ll >= Rl;
  const double Lr = 0.5 * fmax(u, 0.0) * fmax(u, 0.0);
  const double Rr = 0.5 * fmin(ur, 0.0) * fmin(ur, 0.0);
  const bool tr = Lr >= Rr;
  const double Fl = tl ? Ll : Rl, Fr = tr ? Lr : Rr;
  const double inv_dx2 = inv_dx * inv_dx;
  StencilRow o;
  o.fnu = (ur - 2.0 * u + ul) * inv_dx2;
  o.f = -(Fr - Fl) * inv_dx + nu * o.fnu;
  const double dFl_dl = tl ? fmax(ul, 0.0) : 0.0;
  const double dFl_dc = tl ? 0.0 : fmin(u, 0.0);
  const double dFr_dc = tr ? fmax(u, 0.0) : 0.0;
  const double dFr_dr = tr ? 0.0 : fmin(ur, 0.0);
  o.dl = dFl_dl * inv_dx + nu * inv_dx2;
  o.dc = (dFl_dc - dFr_dc) * inv_dx - 2.0 * nu * inv_dx2;
  o.dr = -dFr_dr * inv_dx + nu * inv_dx2;
  return o;
}

}  // namespace rom
