"""Mutation check of the oracle's pins.

Each entry below plants one plausible mistake (a flipped sign, a dropped term, a
transposed index or operand, a wrong constant) in a private copy of the oracle
under a temporary directory, and the oracle's pin suite (the tests/test_oracle_*
files, which check the oracle against closed forms, brute force, finite
differences and the paper's printed values, never against the CUDA path) must
fail on that copy.  The unmodified copy must pass, which also shows that the
copies, not the oracle in this repository, are the ones under test.

Mistakes that leave the arithmetic unchanged for every input the method can see
are not listed: the moment matrix D_p of the quadratic B-spline is (dx^2/4) I,
so B_p D_p^-1 and D_p^-1 B_p agree; the Cauchy stress is symmetric, so
sigma_ab grad_b and sigma_ba grad_b agree; the walls in plain index order
already put the floor after every wall that can share a node with it; and the
adjoint's own mass threshold is unobservable, since a node below it affects the
result in proportion to its weight, about 1e-13.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")

# pin files, cheapest first (each run stops at its first failure)
C_PINS = ["test_oracle_bspline.py", "test_oracle_transfers.py", "test_oracle_transfer.py",
          "test_oracle_boundary.py", "test_oracle_constitutive.py", "test_oracle_obstacles.py",
          "test_oracle_adjoint.py", "test_oracle_adjoint_dp.py", "test_oracle_inverse_velocity.py",
          "test_oracle_hydrostatic.py"]
MLP_PINS = ["test_oracle_mlp.py"]
MONITOR_PINS = ["test_oracle_inverse_velocity.py"]     # the reverse recursion of the velocity problems

C = "mpm_oracle.c"
VI = "velocity_inverse_oracle.py"
# where each mutated file lives
HOME = {C: "oracle", "mlp.py": "oracle", "__init__.py": "oracle", VI: "tests"}
# (name, file, text, replacement, occurrence of text to replace)
MUTANTS = [
    # quadratic B-spline (Sec. 2.1)
    ("phi_bar centre constant", C, "return -a * a + 0.75;", "return -a * a + 0.7;", 0),
    ("phi_bar outer constant", C, "return 0.5 * a * a - 1.5 * a + 9.0 / 8.0;", "return 0.5 * a * a - 1.5 * a + 1.0;", 0),
    ("dphi_bar outer sign", C, "if (a < 1.5) return s * (a - 1.5);", "if (a < 1.5) return (a - 1.5);", 0),
    ("stencil base without the half-cell shift", C, "base[a] = (int)floor(xp[a] / P->dx - 0.5);",
     "base[a] = (int)floor(xp[a] / P->dx);", 0),
    ("stencil node coordinate one cell off", C, "S->xi[k][a] = cell * P->dx;", "S->xi[k][a] = (cell + 1) * P->dx;", 0),
    ("weight gradient with derivative factors", C, "for (int b = 0; b < d; ++b) if (b != a) g *= fa[b];",
     "for (int b = 0; b < d; ++b) if (b != a) g *= dfa[b];", 0),
    ("node index axes transposed", C, "for (int a = P->dim - 1; a >= 0; --a) idx = idx * nodes_axis(P, a) + j[a];",
     "for (int a = 0; a < P->dim; ++a) idx = idx * nodes_axis(P, a) + j[a];", 0),
    ("moment matrix without the weight", C, "D[a * d + b] += S->phi[k] * (S->xi[k][a] - xp[a])",
     "D[a * d + b] += (S->xi[k][a] - xp[a])", 0),
    # P2G (Sec. 2.2)
    ("P2G mass without the weight", C, "gm[i] += mp * phi;", "gm[i] += mp;", 0),
    ("P2G affine matrix transposed", C, "aff += M[a * d + b] * (S.xi[k][b] - xp[b]);",
     "aff += M[b * d + a] * (S.xi[k][b] - xp[b]);", 0),
    ("P2G affine term dropped", C, "gq[i * d + a] += phi * mp * (vp[a] + aff);", "gq[i * d + a] += phi * mp * vp[a];", 0),
    ("P2G internal force sign", C, "gf[i * d + a] += -Vp * fint + phi * mp * P->gravity[a];",
     "gf[i * d + a] += Vp * fint + phi * mp * P->gravity[a];", 0),
    ("P2G gravity dropped", C, "gf[i * d + a] += -Vp * fint + phi * mp * P->gravity[a];",
     "gf[i * d + a] += -Vp * fint;", 0),
    ("P2G volume from the initial volume", C, "double Vp = mp / rho[p];", "double Vp = P->particle_volume;", 0),
    ("P2G force with the stress trace", C, "fint += S.grad[k][b] * sp[b * 3 + a];",
     "fint += S.grad[k][a] * sp[b * 3 + b];", 0),
    # Coulomb wall contact (Eq. coulomb_friction)
    ("friction on separating nodes", C, "if (dvn <= 0.0) return;", "if (dvn < -1e300) return;", 0),
    ("friction without the stick cap", C, "mup = cn / dvn < mu ? cn / dvn : mu;", "mup = mu;", 0),
    ("friction tangential sign", C, "out[a] = v[a] - dvn * (n[a] + mup * nxw[a]);",
     "out[a] = v[a] - dvn * (n[a] - mup * nxw[a]);", 0),
    ("friction keeps the normal velocity", C, "out[a] = v[a] - dvn * (n[a] + mup * nxw[a]);",
     "out[a] = v[a] - dvn * (mup * nxw[a]);", 0),
    ("friction segment index transposed", C, "return P->mu[w][s[1] * P->n_seg[w][0] + s[0]];",
     "return P->mu[w][s[0] * P->n_seg[w][1] + s[1]];", 0),
    ("friction segment from the node index", C, "long num = (long)(j[t[q]] - 1) * ns;",
     "long num = (long)(j[t[q]]) * ns;", 0),
    # grid update (Sec. 2.2)
    ("grid update with half the time step", C, "vi[a] = vn + P->dt * an;", "vi[a] = vn + 0.5 * P->dt * an;", 0),
    ("walls only on ghost nodes", C, "int on_wall = hi ? (coord >= L) : (coord <= 0.0);",
     "int on_wall = hi ? (coord > L) : (coord < 0.0);", 0),
    ("wall normal inward", C, "nrm[a] = hi ? 1.0 : -1.0;", "nrm[a] = hi ? -1.0 : 1.0;", 0),
    ("floor wall first", C, "for (int w = 0; w < 2 * d; ++w) if (w != floor_w) order[nw++] = w;\n"
     "    order[nw++] = floor_w;", "order[nw++] = floor_w;\n"
     "    for (int w = 0; w < 2 * d; ++w) if (w != floor_w) order[nw++] = w;", 0),
    # rigid obstacles (Sec. 4.1)
    ("obstacle normal inward", C, "nrm[best / 2] = (best % 2) ? 1.0 : -1.0;", "nrm[best / 2] = (best % 2) ? -1.0 : 1.0;", 0),
    ("obstacle contact on separating nodes", C, "if (!(vn < 0.0)) return 0;", "if (!(vn > 0.0)) return 0;", 0),
    ("obstacle faces on the domain boundary", C, "if (lo > 0 && (best < 0 || c - lo < best_dist))",
     "if (lo >= 0 && (best < 0 || c - lo < best_dist))", 0),
    ("obstacle ties to the later face", C, "(best < 0 || hi - c < best_dist)", "(best < 0 || hi - c <= best_dist)", 0),
    # Tait equation of state (Sec. 2.3)
    ("Tait density ratio inverted", C, "pow(rho / P->rho0, P->gamma) - 1.0", "pow(P->rho0 / rho, P->gamma) - 1.0", 0),
    ("Tait without 1/gamma", C, "return P->bulk_K / P->gamma * (pow(", "return P->bulk_K * (pow(", 0),
    # Drucker-Prager constants and update (Appendix A)
    ("bulk modulus", C, "c->K = P->E / (3.0 * (1.0 - 2.0 * P->nu));", "c->K = P->E / (3.0 * (1.0 - P->nu));", 0),
    ("shear modulus", C, "c->G = P->E / (2.0 * (1.0 + P->nu));", "c->G = P->E / (1.0 + P->nu);", 0),
    ("q_phi of the extension cone", C, "c->q_phi = 6.0 * sin(phi) / (sqrt(3.0) * (3.0 + sin(phi)));",
     "c->q_phi = 6.0 * sin(phi) / (sqrt(3.0) * (3.0 - sin(phi)));", 0),
    ("k_phi with sin", C, "c->k_phi = 6.0 * P->cohesion * cos(phi)", "c->k_phi = 6.0 * P->cohesion * sin(phi)", 0),
    ("q_psi from the friction angle", C, "c->q_psi = 6.0 * sin(psi) / (sqrt(3.0) * (3.0 + sin(psi)));",
     "c->q_psi = 6.0 * sin(phi) / (sqrt(3.0) * (3.0 + sin(phi)));", 0),
    ("alpha_P sign", C, "c->alpha_P = sqrt(1.0 + c->q_phi * c->q_phi) - c->q_phi;",
     "c->alpha_P = sqrt(1.0 + c->q_phi * c->q_phi) + c->q_phi;", 0),
    ("tau_P sign", C, "c->tau_P = c->k_phi - c->q_phi * c->sig_t;", "c->tau_P = c->k_phi + c->q_phi * c->sig_t;", 0),
    ("tension cutoff not capped by the cone apex", C,
     "if (c->q_phi > 0.0 && c->k_phi / c->q_phi < c->sig_t) c->sig_t = c->k_phi / c->q_phi;", "", 0),
    ("Jaumann term sign", C, "v += s[i * 3 + k] * dw[j * 3 + k] + s[j * 3 + k] * dw[i * 3 + k];",
     "v += s[i * 3 + k] * dw[j * 3 + k] - s[j * 3 + k] * dw[i * 3 + k];", 0),
    ("Jaumann rotation dropped", C, "v += s[i * 3 + k] * dw[j * 3 + k] + s[j * 3 + k] * dw[i * 3 + k];",
     "v += 0.0 * (s[i * 3 + k] * dw[j * 3 + k] + s[j * 3 + k] * dw[i * 3 + k]);", 0),
    ("elastic tensor without minor symmetry", C,
     "double C = lam * (i == j) * (k == l) + c.G * ((i == k) * (j == l) + (i == l) * (j == k));",
     "double C = lam * (i == j) * (k == l) + c.G * ((i == k) * (j == l));", 0),
    ("Lame lambda", C, "double lam = c.K - 2.0 * c.G / 3.0;", "double lam = c.K - c.G / 3.0;", 0),
    ("tau without the half", C, "double tau = sqrt(0.5 * ss);", "double tau = sqrt(ss);", 0),
    ("shear yield sign of the mean stress", C, "double fs = tau - c.k_phi + c.q_phi * sm;",
     "double fs = tau - c.k_phi - c.q_phi * sm;", 0),
    ("zone I without the tension check", C, "if (fs <= 0.0 && ft < 0.0) {", "if (fs <= 0.0) {", 0),
    ("zone II multiplier with q_phi twice", C, "double dl = fs / (c.G + c.K * c.q_phi * c.q_psi);",
     "double dl = fs / (c.G + c.K * c.q_phi * c.q_phi);", 0),
    ("zone II mean stress return sign", C, "double sm_n = sm - c.K * c.q_psi * dl;",
     "double sm_n = sm + c.K * c.q_psi * dl;", 0),
    ("zone II equivalent plastic strain", C, "*eps += dl * sqrt(1.0 / 3.0 + 2.0 / 9.0 * c.q_psi * c.q_psi);",
     "*eps += dl;", 0),
    ("zone II corner guard dropped", C, "if (!P->dp_literal && sm_n > c.sig_t) {",
     "if (0 && sm_n > c.sig_t) {", 0),
    ("zone III mean stress sign", C, "s[q] = st[q] + (q % 4 == 0 ? (c.sig_t - sm) : 0.0);",
     "s[q] = st[q] + (q % 4 == 0 ? (sm - c.sig_t) : 0.0);", 0),
    ("zone III equivalent plastic strain", C, "*eps += sqrt(2.0) / 3.0 * dlt;", "*eps += dlt;", 0),
    ("zone III corner guard dropped", C, "if (!P->dp_literal && tau > c.tau_P) {", "if (0 && tau > c.tau_P) {", 0),
    # G2P (Sec. 2.2, Appendix B)
    ("G2P affine matrix transposed", C, "Bp[a * d + b] += S.phi[k] * vi[a] * (S.xi[k][b] - xp[b]);",
     "Bp[a * d + b] += S.phi[k] * vi[b] * (S.xi[k][a] - xp[a]);", 0),
    ("G2P velocity gradient transposed", C, "L[a * d + b] += vi[a] * S.grad[k][b];",
     "L[a * d + b] += vi[b] * S.grad[k][a];", 0),
    ("G2P position not clamped at the top", C, "if (xn > Lmax) xn = Lmax;", "", 0),
    ("deformation gradient multiplied on the right", C, "matmul(d, A, F + p * d * d, Fn);",
     "matmul(d, F + p * d * d, A, Fn);", 0),
    ("density update sign", C, "rho[p] = rho[p] / (1.0 + trdd);", "rho[p] = rho[p] * (1.0 + trdd);", 0),
    ("strain increment without the half", C, "dd[a * 3 + b] = 0.5 * (L[a * d + b] + L[b * d + a]) * dt;",
     "dd[a * 3 + b] = (L[a * d + b] + L[b * d + a]) * dt;", 0),
    ("spin increment sign", C, "dw[a * 3 + b] = 0.5 * (L[a * d + b] - L[b * d + a]) * dt;",
     "dw[a * 3 + b] = 0.5 * (L[b * d + a] - L[a * d + b]) * dt;", 0),
    ("viscous stress without the bulk correction", C,
     "sp[a * 3 + b] = (a == b ? -pr - 2.0 / 3.0 * mu * tr_rate : 0.0) + 2.0 * mu * rate;",
     "sp[a * 3 + b] = (a == b ? -pr : 0.0) + 2.0 * mu * rate;", 0),
    ("FLIP increment sign", C, "vflip[a] = vp[a] + P->flip_alpha * (v[p * d + a] - vo[a]);",
     "vflip[a] = vp[a] + P->flip_alpha * (vo[a] - v[p * d + a]);", 0),
    ("TPIC keeps the affine matrix", C,
     "B[p * d * d + q] = P->transfer == 1 ? L[q] : (P->transfer >= 2 ? 0.0 : Bp[q]);",
     "B[p * d * d + q] = P->transfer >= 2 ? 0.0 : Bp[q];", 0),
    ("C_p without the inverse moment matrix", C, "matmul(d, B + p * d * d, Dinv, C + p * d * d);",
     "for (int q = 0; q < d * d; ++q) C[p * d * d + q] = B[p * d * d + q];", 0),
    ("FLIP old grid velocity is momentum", C, "gvo[i * d + a] = gm[i] > m_eps ? gq[i * d + a] / gm[i] : 0.0;",
     "gvo[i * d + a] = gm[i] > m_eps ? gq[i * d + a] : 0.0;", 0),
    # one-step adjoint (Sec. 3.1)
    ("Hessian of the centre piece", C, "ddf[a] = (ax < 0.5 ? -2.0 : (ax < 1.5 ? 1.0 : 0.0))",
     "ddf[a] = (ax < 0.5 ? 2.0 : (ax < 1.5 ? 1.0 : 0.0))", 0),
    ("wall adjoint slide term sign", C, "ib[a] = s * obt[a] - mu * dot * (n[a] / vtn - vn * vt[a] / (vtn * vtn * vtn));",
     "ib[a] = s * obt[a] + mu * dot * (n[a] / vtn - vn * vt[a] / (vtn * vtn * vtn));", 0),
    ("wall adjoint friction gradient sign", C, "if (mub) *mub += -dot * vn / vtn;", "if (mub) *mub += dot * vn / vtn;", 0),
    ("wall adjoint passes through stick", C, "if (vtn <= mu * vn) { for (int a = 0; a < 3; ++a) ib[a] = 0.0; return; }",
     "if (vtn <= mu * vn) { for (int a = 0; a < 3; ++a) ib[a] = obt[a]; return; }", 0),
    ("adjoint segment index transposed", C, "return s[1] * P->n_seg[w][0] + s[0];",
     "return s[0] * P->n_seg[w][1] + s[1];", 0),
    ("Tait derivative exponent", C, "pow(rho / P->rho0, P->gamma - 1.0)", "pow(rho / P->rho0, P->gamma)", 0),
    ("adjoint through the position clamp", C, "xb0[p * d + a] = clamped ? 0.0 : xb1[p * d + a];",
     "xb0[p * d + a] = xb1[p * d + a];", 0),
    ("adjoint of the density update sign", C, "double trLb = -rhob1[p] * rho[p] * dt / (den * den);",
     "double trLb = rhob1[p] * rho[p] * dt / (den * den);", 0),
    ("adjoint spin part sign", C,
     "Lb[a * d + b] = 0.5 * dt * (ddb[a * 3 + b] + ddb[b * 3 + a] + dwb[a * 3 + b] - dwb[b * 3 + a]);",
     "Lb[a * d + b] = 0.5 * dt * (ddb[a * 3 + b] + ddb[b * 3 + a] + dwb[b * 3 + a] - dwb[a * 3 + b]);", 0),
    ("adjoint G2P affine matrix transposed", C, "for (int b = 0; b < d; ++b) Br += Bb[a * d + b] * r[b];",
     "for (int b = 0; b < d; ++b) Br += Bb[b * d + a] * r[b];", 0),
    ("adjoint G2P position term from B sign", C, "xb0[p * d + b] += -Bb[a * d + b] * phi * via;",
     "xb0[p * d + b] += Bb[a * d + b] * phi * via;", 0),
    ("adjoint G2P Hessian term dropped", C, "xb0[p * d + b] += phib * S.grad[k][b] + hb;",
     "xb0[p * d + b] += phib * S.grad[k][b];", 0),
    ("adjoint P2G Hessian term dropped", C, "xb0[p * d + b] += phib * S.grad[k][b] + hb;",
     "xb0[p * d + b] += phib * S.grad[k][b];", 1),
    ("adjoint G2P grid term without B", C, "gvb[i * 3 + a] += phi * vbt[a] + phi * Br + Lg;",
     "gvb[i * 3 + a] += phi * vbt[a] + Lg;", 0),
    ("adjoint G2P position without dt", C, "vbt[a] = vb1[p * d + a] + (clamped ? 0.0 : dt * xb1[p * d + a]);",
     "vbt[a] = vb1[p * d + a] + (clamped ? 0.0 : xb1[p * d + a]);", 0),
    ("adjoint grid mass sign", C, "gmb[i] += -ob[a] * (gq[i * d + a] + dt * gf[i * d + a]) / (gm[i] * gm[i]);",
     "gmb[i] += ob[a] * (gq[i * d + a] + dt * gf[i * d + a]) / (gm[i] * gm[i]);", 0),
    ("adjoint grid force without dt", C, "gfb[i * d + a] = dt * ob[a] / gm[i];", "gfb[i * d + a] = ob[a] / gm[i];", 0),
    ("adjoint obstacle projection skipped", C, "for (int b = 0; b < 3; ++b) ob[b] -= obn * onrm[o][b];",
     "for (int b = 0; b < 3; ++b) ob[b] -= 0.0 * obn * onrm[o][b];", 0),
    ("adjoint P2G affine position term sign", C, "xb0[p * d + b] += -phi * mp * qb * M[a * d + b];",
     "xb0[p * d + b] += phi * mp * qb * M[a * d + b];", 0),
    ("adjoint P2G gravity term dropped", C, "phib += mp * qb * qa + mp * fb * P->gravity[a];",
     "phib += mp * qb * qa;", 0),
    ("adjoint P2G stress sign", C, "sigb0[p * 9 + a * 3 + b] += -Vp * S.grad[k][b] * fb;",
     "sigb0[p * 9 + a * 3 + b] += Vp * S.grad[k][b] * fb;", 0),
    ("adjoint P2G pressure sign", C, "prb += Vp * fb * S.grad[k][a];", "prb += -Vp * fb * S.grad[k][a];", 0),
    ("adjoint P2G without the inverse moment matrix", C, "Bb0[p * d * d + a * d + b] = s;",
     "Bb0[p * d * d + a * d + b] = Mb[a * d + b];", 0),
    ("adjoint P2G volume sign", C, "rhob0[p] += Vb * (-mp / (rho[p] * rho[p]))", "rhob0[p] += Vb * (mp / (rho[p] * rho[p]))", 0),
    ("adjoint P2G mass term dropped", C, "double phib = mp * gmb[i], gradb[3] = {0, 0, 0};",
     "double phib = 0.0, gradb[3] = {0, 0, 0};", 0),
    ("Hessian mixed term on the diagonal", C, "h *= na == 0 ? f[c] : (na == 1 ? df[c] : ddf[c]);",
     "h *= na == 0 ? f[c] : df[c];", 0),
    ("Hessian of the outer piece", C, "(ax < 1.5 ? 1.0 : 0.0)", "(ax < 1.5 ? -1.0 : 0.0)", 0),
    ("wall adjoint without the tangential projection", C, "for (int a = 0; a < 3; ++a) obt[a] = ob[a] - obn * n[a];",
     "for (int a = 0; a < 3; ++a) obt[a] = ob[a];", 0),
    ("wall adjoint slide scale sign", C, "double s = 1.0 - mu * vn / vtn;", "double s = 1.0 + mu * vn / vtn;", 0),
    ("wall adjoints in forward order", C, "for (int q = nw - 1; q >= 0; --q) {", "for (int q = 0; q < nw; ++q) {", 0),
    ("wall adjoint linearised at the wall's output", C, "wall_vjp(chain[q], nrm, wall_mu(P, w, j), ob, ib, mub);",
     "wall_vjp(chain[q + 1], nrm, wall_mu(P, w, j), ob, ib, mub);", 0),
    ("adjoint grid momentum without the mass", C, "gqb[i * d + a] = ob[a] / gm[i];", "gqb[i * d + a] = ob[a];", 0),
    ("adjoint P2G velocity without the weight", C, "vb0[p * d + a] += phi * mp * qb;", "vb0[p * d + a] += mp * qb;", 0),
    ("adjoint P2G affine adjoint transposed", C, "Mb[a * d + b] += phi * mp * qb * r[b];",
     "Mb[b * d + a] += phi * mp * qb * r[b];", 0),
    ("adjoint P2G stress gradient index", C, "gradb[b] += -Vp * sp[a * 3 + b] * fb;",
     "gradb[a] += -Vp * sp[a * 3 + b] * fb;", 0),
    ("adjoint P2G sand volume sign", C, "Vb += -sp[a * 3 + b] * S.grad[k][b] * fb;",
     "Vb += sp[a * 3 + b] * S.grad[k][b] * fb;", 0),
    ("adjoint P2G fluid gradient sign", C, "gradb[a] += Vp * pr * fb;", "gradb[a] += -Vp * pr * fb;", 0),
    ("adjoint P2G fluid volume dropped", C, "Vb += pr * fb * S.grad[k][a];", "Vb += 0.0 * pr * fb * S.grad[k][a];", 0),
    ("adjoint G2P gradient adjoint transposed", C, "gradb[b] += Lb[a * d + b] * via;",
     "gradb[b] += Lb[b * d + a] * via;", 0),
    ("adjoint G2P velocity-gradient term transposed", C, "Lg += Lb[a * d + b] * S.grad[k][b];",
     "Lg += Lb[b * d + a] * S.grad[k][b];", 0),
    ("adjoint G2P weight term without B", C, "phib += vbt[a] * via + Br * via;", "phib += vbt[a] * via;", 0),
    ("adjoint density carried without the update", C, "rhob0[p] = rhob1[p] / den;", "rhob0[p] = rhob1[p];", 0),
    ("obstacle extent rounded down", C, "long lo = (long)ceil(P->obstacle[o][0][a] / P->dx - 1e-9);",
     "long lo = (long)floor(P->obstacle[o][0][a] / P->dx);", 0),
    ("obstacle high side open", C, "if (c < lo || c > hi) return 0;", "if (c < lo || c >= hi) return 0;", 0),
    ("segment beyond the far wall", C, "if (sq > ns - 1) sq = ns - 1;", "if (sq > ns - 1) sq = ns > 1 ? ns - 2 : 0;", 0),
    ("adjoint segment beyond the far wall", C, "if (sq > ns - 1) sq = ns - 1;",
     "if (sq > ns - 1) sq = ns > 1 ? ns - 2 : 0;", 1),
    ("mass threshold scale", C, "double m_eps = 1e-10 * P->rho0 * pow(P->dx, d);",
     "double m_eps = 1e-10 / P->rho0 * pow(P->dx, d);", 0),
    ("floor index in 3D", C, "int floor_w = 2 * (d - 1);", "int floor_w = 2 / (d - 1);", 0),
    ("adjoint floor index in 3D", C, "nw = 0, floor_w = 2 * (d - 1);", "nw = 0, floor_w = 2 / (d - 1);", 0),
    ("zone III corner mean stress sign", C, "s[q] = r * sdev[q] + (q % 4 == 0 ? c.sig_t : 0.0);",
     "s[q] = r * sdev[q] - (q % 4 == 0 ? c.sig_t : 0.0);", 0),
    ("adjoint clamp test at the top", C, "int clamped = xn < 0.0 || xn > P->n_cells[a] * P->dx;",
     "int clamped = xn < 0.0 || xn > P->n_cells[a] / P->dx;", 0),
    ("adjoint obstacle projection on a y face", C,
     "double obn = ob[0] * onrm[o][0] + ob[1] * onrm[o][1] + ob[2] * onrm[o][2];",
     "double obn = ob[0] * onrm[o][0] - ob[1] * onrm[o][1] + ob[2] * onrm[o][2];", 0),
    ("adjoint zone II/III line", C, "double h = tau - c.tau_P - c.alpha_P * (sm - c.sig_t);",
     "double h = tau - c.tau_P - c.alpha_P / (sm - c.sig_t);", 1),
    # Drucker-Prager adjoint (Appendix A, reverse)
    ("DP adjoint corner keeps the mean-stress path", C, "double sm_nb = corner ? 0.0 : trb;", "double sm_nb = trb;", 0),
    ("DP adjoint corner keeps the tau path", C, "if (!corner) tau_nb = rb / tau;", "tau_nb = rb / tau;", 0),
    ("DP adjoint cone slope sign", C, "sm_nb += -c.q_phi * tau_nb;", "sm_nb += c.q_phi * tau_nb;", 0),
    ("DP adjoint zone III corner sign", C, "taub += -rb * c.tau_P / (tau * tau);", "taub += rb * c.tau_P / (tau * tau);", 0),
    ("DP adjoint Jaumann stress index", C, "sb0[j * 3 + k] += g * dw[i * 3 + k];", "sb0[j * 3 + k] += g * dw[k * 3 + i];", 0),
    ("DP adjoint mean without the third", C, "for (int a = 0; a < 3; ++a) stb[a * 4] += smb / 3.0;",
     "for (int a = 0; a < 3; ++a) stb[a * 4] += smb;", 0),
    ("DP adjoint zone II mean-stress chain", C, "smb += sm_nb * (1.0 - c.K * c.q_psi * c.q_phi / A);",
     "smb += sm_nb;", 0),
    ("DP adjoint zone II tau chain sign", C, "taub += sm_nb * (-c.K * c.q_psi / A);", "taub += sm_nb * (c.K * c.q_psi / A);", 0),
    ("DP adjoint radial scale sign", C, "taub += -rb * tau_n / (tau * tau);", "taub += rb * tau_n / (tau * tau);", 0),
    ("DP adjoint zone III mean sign", C, "smb += -trb;", "smb += trb;", 0),
    ("DP adjoint Jaumann index", C, "dwb[j * 3 + k] += g * s[i * 3 + k];", "dwb[k * 3 + j] += g * s[i * 3 + k];", 0),
    ("DP adjoint elastic tensor", C, "c.G * (stb[k * 3 + l] + stb[l * 3 + k]);", "c.G * stb[k * 3 + l];", 0),
    ("DP adjoint tau derivative", C, "sdevb[q] += taub * 0.5 * sdev[q] / tau;", "sdevb[q] += taub * sdev[q] / tau;", 0),
    ("DP adjoint deviator trace", C, "smb += -sdev_tr;", "smb += sdev_tr;", 0),
    # warm-start network (oracle/mlp.py)
    ("GELU scale", "mlp.py", "_erf(z / math.sqrt(2.0)))\n", "_erf(z / 2.0))\n", 0),
    ("GELU derivative exponent", "mlp.py", "np.exp(-0.5 * z * z)", "np.exp(-z * z)", 0),
    ("bf16 ties away from zero", "mlp.py", "((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16))",
     "((u + np.uint64(0x8000)) >> np.uint64(16))", 0),
    ("output range without the lower bound", "mlp.py", "return lo + (hi - lo) * s, xs, zs", "return lo + hi * s, xs, zs", 0),
    ("bias gradient averaged", "mlp.py", "gb = dz.sum(axis=0)", "gb = dz.mean(axis=0)", 0),
    ("squared-error gradient without the 2", "mlp.py", "backward(params, widths, x, 2.0 * e / n,",
     "backward(params, widths, x, e / n,", 0),
    ("backward through unrounded weights", "mlp.py", "da = dzr @ r(W)", "da = dz @ W", 0),
    ("hidden activations not rounded", "mlp.py", "xs.append(r(act(z)))", "xs.append(act(z))", 0),
    ("network input not rounded", "mlp.py", "xs, zs = [r(x)], []", "xs, zs = [np.asarray(x, dtype=np.float64)], []", 0),
    ("weight gradient from the unrounded error", "mlp.py", "gW = dzr.T @ xs[l]", "gW = dz.T @ xs[l]", 0),
    ("output sigmoid derivative sign", "mlp.py", "dz = np.asarray(dy, dtype=np.float64) * (hi - lo) * s * (1.0 - s)",
     "dz = np.asarray(dy, dtype=np.float64) * (hi - lo) * s * (1.0 + s)", 0),
    ("ReLU derivative 1 at zero", "mlp.py", "(np.asarray(z) > 0.0)", "(np.asarray(z) >= 0.0)", 0),
    ("leaky ReLU", "mlp.py", "return np.maximum(z, 0.0)", "return np.maximum(z, 0.01 * z)", 0),
    ("linear output scaled like a sigmoid", "mlp.py", "dz = np.asarray(dy, dtype=np.float64)\n    else:",
     "dz = 0.25 * np.asarray(dy, dtype=np.float64)\n    else:", 0),
    ("backward through GELU whatever the hidden activation", "mlp.py", "dact = _ACT[hidden][1]",
     "dact = _ACT['gelu'][1]", 0),
    # velocity monitors (oracle/__init__.py)
    ("monitor box open at the top", "__init__.py", "inside = np.all((x >= np.asarray(lo, dtype=np.float64)) & "
     "(x <= np.asarray(hi, dtype=np.float64)), axis=1)\n        cnt[l]",
     "inside = np.all((x >= np.asarray(lo, dtype=np.float64)) & (x < np.asarray(hi, dtype=np.float64)), axis=1)\n"
     "        cnt[l]", 0),
    ("monitor mean over all particles", "__init__.py", "Q[l] = v[inside].sum(axis=0) / cnt[l]",
     "Q[l] = v[inside].sum(axis=0) / len(x)", 0),
    ("monitor seed without the count", "__init__.py", "g[inside] += 2.0 * e / cnt[l]", "g[inside] += 2.0 * e", 0),
    # parameters handed to the C step (oracle/__init__.py)
    ("segment counts swapped", "__init__.py", "P.n_seg[wall][0], P.n_seg[wall][1] = int(nseg[0]), int(nseg[1])",
     "P.n_seg[wall][0], P.n_seg[wall][1] = int(nseg[1]), int(nseg[0])", 0),
    ("obstacle corners swapped", "__init__.py", "P.obstacle[o][0][a] = float(lo[a])\n"
     "                P.obstacle[o][1][a] = float(hi[a])", "P.obstacle[o][0][a] = float(hi[a])\n"
     "                P.obstacle[o][1][a] = float(lo[a])", 0),
    ("particle mass is the volume", C, "{ return P->rho0 * P->particle_volume; }", "{ return P->particle_volume; }", 0),
    # reverse recursion of the initial-velocity problems (tests/velocity_inverse_oracle.py)
    ("tracked seed without the 2", VI, "lam[0][ids] += 2.0 * e", "lam[0][ids] += e", 0),
    ("step adjoint taken at the later state", VI, "lam, _ = orc.step_vjp(states[t - 1], *lam)",
     "lam, _ = orc.step_vjp(states[t], *lam)", 0),
    ("initial adjoint of the position returned", VI, "return loss, lam[1]", "return loss, lam[0]", 0),
    ("monitor seed dropped", VI, "lam[1] += g", "lam[1] += 0.0 * g", 0),
]


def _pins(fname):
    return {C: C_PINS, "mlp.py": MLP_PINS, "__init__.py": C_PINS, VI: MONITOR_PINS}[fname]


def _replace_nth(src: str, old: str, new: str, nth: int) -> str:
    at = -1
    for _ in range(nth + 1):
        at = src.find(old, at + 1)
        if at < 0:
            raise ValueError(f"text not found (occurrence {nth}): {old!r}")
    return src[:at] + new + src[at + len(old):]


def _tree(base: str, mutant=None) -> str:
    """A private copy of the oracle and its pin files under base, with one mistake planted."""
    files = [("oracle", f) for f in ("__init__.py", "mlp.py", "mpm_oracle.c")]
    files += [("tests", f) for f in sorted(os.listdir(TESTS))
              if f.startswith("test_oracle_") and f.endswith(".py") and f != os.path.basename(__file__)
              or f in ("conftest.py", VI)]
    for d in ("oracle", "tests"):
        os.makedirs(os.path.join(base, d))
    for d, f in files:
        with open(os.path.join(ROOT, d, f)) as fh:
            src = fh.read()
        if mutant is not None and mutant[1] == f and HOME[f] == d:
            src = _replace_nth(src, mutant[2], mutant[3], mutant[4])
        with open(os.path.join(base, d, f), "w") as fh:
            fh.write(src)
    shutil.copytree(os.path.join(TESTS, "golden"), os.path.join(base, "tests", "golden"))
    os.symlink(os.path.join(ROOT, "paper_2507_04192_gb300"), os.path.join(base, "paper_2507_04192_gb300"))
    with open(os.path.join(base, "pytest.ini"), "w") as fh:
        fh.write("[pytest]\naddopts = -p no:cacheprovider\n")
    return base


def _env():
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env["PYTHONDONTWRITEBYTECODE"] = "1"
    return env


def _run(base: str, pins) -> subprocess.CompletedProcess:
    """Build the copy's oracle, then run its pins; returns the pytest process."""
    env = _env()
    b = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.build(force=True))"], cwd=base, env=env,
                       capture_output=True, text=True, timeout=300)
    if b.returncode != 0 or not b.stdout.strip().startswith(base):
        raise RuntimeError(f"oracle copy did not build under {base}: {b.stdout[-500:]} {b.stderr[-2000:]}")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu"] +
                          [os.path.join("tests", p) for p in pins], cwd=base, env=env,
                          capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def outcomes():
    """Runs the unmodified copy and every mutant (in parallel) once per module."""
    with tempfile.TemporaryDirectory(prefix="oracle_mut_") as tmp:
        def one(k):
            base = _tree(os.path.join(tmp, f"m{k}"), None if k < 0 else MUTANTS[k])
            pins = C_PINS + MLP_PINS if k < 0 else _pins(MUTANTS[k][1])
            return k, _run(base, pins)

        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            res = dict(ex.map(one, range(-1, len(MUTANTS))))
    return res


def test_unmodified_copy_passes(outcomes):
    r = outcomes[-1]
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("k", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(outcomes, k):
    r = outcomes[k]
    # 1 = a pin failed; anything else (0 = survived, 2+ = the copy did not import) is a harness problem
    assert r.returncode == 1, f"{MUTANTS[k][0]}: exit {r.returncode}\n{r.stdout[-2000:]}{r.stderr[-1000:]}"
