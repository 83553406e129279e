"""Planted-mistake check of the oracle's pins (test infrastructure, no GPU).

Each entry below is a plausible mistake in ``oracle.c``: a dropped term, a
wrong sign, index or spacing, a swapped operand, a rule applied to the wrong
variable.  ``python oracle/mutants.py`` copies the oracle into a temporary
directory once per mistake, plants it, and runs every CPU pin of the oracle
(``tests/test_oracle_*.py`` and ``tests/test_workloads.py``) against the
copy.  A mistake that no pin catches is reported.  Two are known and
accepted: the Chakravarthy limiter's coefficient, which is not a default and
is taken as printed in Table 4.2, and which spacing scales the normal
cut-off of the CSF curvature on grids whose spacings differ (every workload
grid has equal spacings).

    python oracle/mutants.py [-j JOBS] [NAME ...]
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ACCEPTED = {"lim_chak", "grad_eps_dxmax"}

# (name, [(text in oracle.c, replacement), ...]); each text occurs once
MUTANTS = [
    ('R_ps_left', [('ps = 0.5 * (pL + pR);                                            /* Eq. 3-1 */',
      'ps = pL;')]),
    ('R_us_sign', [('us = (rL * cL * uL + rR * cR * uR + pL - pR + J) / (rL * cL + rR * cR); /* Eq. 3-2 */',
      'us = (rL * cL * uL + rR * cR * uR - pL + pR + J) / (rL * cL + rR * cR);')]),
    ('R_imp_swap', [('us = (rL * cL * uL + rR * cR * uR + pL - pR + J) / (rL * cL + rR * cR); /* Eq. 3-2 */',
      'us = (rR * cR * uL + rL * cL * uR + pL - pR + J) / (rL * cL + rR * cR);')]),
    ('D_IL_swap', [('double IL = (3.0 * rho4[1] + rho4[2]) * cm / 4.0;',
      'double IL = (rho4[1] + 3.0 * rho4[2]) * cm / 4.0;')]),
    ('D_IR_swap', [('double IR = (rho4[1] + 3.0 * rho4[2]) * cm / 4.0;',
      'double IR = (3.0 * rho4[1] + rho4[2]) * cm / 4.0;')]),
    ('D_cm_min', [('double cm = fmax(c4[1], c4[2]);',
      'double cm = fmin(c4[1], c4[2]);')]),
    ('D_us_nod3', [('us = uL - (d3 - J) / (IL + IR);',
      'us = uL - (0.0 * d3 - J) / (IL + IR);')]),
    ('D_f_ps_left', [('            ps = 0.5 * (pL + pR);\n        } else {',
      '            ps = pL;\n        } else {')]),
    ('D_f_us_sign', [('us = (IL * uL + IR * uR + pL - pR + J) / (IL + IR);',
      'us = (IL * uL + IR * uR - pL + pR + J) / (IL + IR);')]),
    ('up_W_swap', [('const double* Ws = (us >= 0.0) ? WL : WR;',
      'const double* Ws = (us >= 0.0) ? WR : WL;')]),
    ('up_rho_swap', [('double rs = (us >= 0.0) ? rL : rR;',
      'double rs = (us >= 0.0) ? rR : rL;')]),
    ('up_e_swap', [('double es = (us >= 0.0) ? eL : eR;',
      'double es = (us >= 0.0) ? eR : eL;')]),
    ('E_no_pu', [('F[1 + nd] = us * rs * (es + ke) + ps * us;',
      'F[1 + nd] = us * rs * (es + ke);')]),
    ('F_ke2', [('for (int a = 0; a < nd; ++a) ke += 0.5 * Ws[a] * Ws[a];',
      'for (int a = 0; a < nd; ++a) ke += Ws[a] * Ws[a];')]),
    ('F_p_dir0', [('(a == d ? ps : 0.0)',
      '(a == 0 ? ps : 0.0)')]),
    ('capj_G_full', [('G[0] = 0.5 * J;',
      'G[0] = J;')]),
    ('capj_Gu', [('G[1] = 0.5 * J * us;',
      'G[1] = 0.0 * J * us;')]),
    ('capj_J_sign', [('(al2[1] - al2[0]) : 0.0;',
      '(al2[0] - al2[1]) : 0.0;')]),
    ('capj_kL', [('P->sigma * 0.5 * (kapL + kapR)',
      'P->sigma * kapL')]),
    ('D1_coef', [('(7.0 * (w2[v] + w3[v]) - w1[v] - w4[v]) / 12.0',
      '(7.0 * (w2[v] + w3[v]) - w1[v] - w4[v]) / 12.5')]),
    ('D1_Y_fourth', [('const int fourth = (v < iY) && !(baro && v == iT);',
      'const int fourth = !(baro && v == iT);')]),
    ('lim_p_koren', [('int lim = (v < nd) ? P->lim_vel : P->lim_scalar;',
      'int lim = (v <= nd) ? P->lim_vel : P->lim_scalar;')]),
    ('cp_ke2', [('        ke += 0.5 * w[a] * w[a];\n    }\n    double e = qc[1 + nd] / rho - ke;',
      '        ke += w[a] * w[a];\n    }\n    double e = qc[1 + nd] / rho - ke;')]),
    ('bc_mirror', [('int s = -1 - i;',
      'int s = -i;')]),
    ('bc_mirror_hi', [('int s = 2 * n - 1 - i;',
      'int s = 2 * n - i;')]),
    ('bc_noflip', [('if (flip[d]) w[d] = -w[d];',
      'if (flip[d] && 0) w[d] = -w[d];')]),
    ('in_T', [('w[nd + 1] = P->in_T;',
      'w[nd + 1] = w[nd + 1];')]),
    ('in_radius', [('<= P->in_radius * P->in_radius',
      '<= 0.81 * P->in_radius * P->in_radius')]),
    ('sens_curl2d', [('double wz = g[1][0] - g[0][1];\n        curl2 = wz * wz;',
      'double wz = g[1][0] + g[0][1];\n        curl2 = wz * wz;')]),
    ('sens_curl3d', [('double wx = g[2][1] - g[1][2]',
      'double wx = g[2][1] + g[1][2]')]),
    ('sens_div', [('for (int a = 0; a < nd; ++a) div += g[a][a];\n    double curl2;',
      'for (int a = 0; a < nd; ++a) div += g[0][a];\n    double curl2;')]),
    ('sens_tg_onesided', [('tg += fabs(ag0 - (1.0 - B->al[bm])) + fabs((1.0 - B->al[bp]) - ag0);',
      'tg += fabs((1.0 - B->al[bp]) - ag0);')]),
    ('sens_and', [('(a5[0] > P->thr_ducros || a5[1] > P->thr_gas || a5[2] > P->thr_vap)',
      '((a5[0] > P->thr_ducros && a5[1] > P->thr_gas) || a5[2] > P->thr_vap)')]),
    ('sens_face_and', [('B.flag[bidx(&B, c[0], c[1], c[2])] > 0.5 ||',
      'B.flag[bidx(&B, c[0], c[1], c[2])] > 0.5 &&')]),
    ('csf_smooth_w', [('static const double w3[3] = {1.0, 2.0, 1.0};',
      'static const double w3[3] = {1.0, 1.0, 1.0};')]),
    ('csf_kappa_sign', [('kappa -= sg * nrm[d] / (scale * P->dx[d]);',
      'kappa += sg * nrm[d] / (scale * P->dx[d]);')]),
    ('csf_galpha_smoothed', [('gu[d] += sg * au / (scale * P->dx[d]);',
      'gu[d] += sg * as / (scale * P->dx[d]);')]),
    ('csf_energy0', [('udg += B->W[(size_t)d * B->cnt + b0] * galpha[d];',
      'udg += 0.0 * galpha[d];')]),
    ('csf_gradeps0', [('if (mag > P->grad_eps / dxmin)',
      'if (mag > 0.0)')]),
    ('hf_pow', [('if (nt < 2) return -Hxx / pow(1.0 + Hx * Hx, 1.5);',
      'if (nt < 2) return -Hxx / pow(1.0 + Hx * Hx, 1.0);')]),
    ('hf_cross', [('- 2.0 * Hxy * Hx * Hy)',
      '+ 2.0 * Hxy * Hx * Hy)')]),
    ('hf_axis_first', [('if (g > gmax) { gsec = gmax; gmax = g; dir = d; }',
      'if (g > gmax && d == 0) { gsec = gmax; gmax = g; dir = d; }')]),
    ('v_transpose', [('double tau = mu * (g[a][d] + g[d][a]);',
      'double tau = mu * (2.0 * g[a][d]);')]),
    ('v_13', [('if (a == d) tau -= 2.0 / 3.0 * mu * div;',
      'if (a == d) tau -= 1.0 / 3.0 * mu * div;')]),
    ('v_heat_sign', [('F[1 + nd] -= utau + kc * dTdx;',
      'F[1 + nd] -= utau - kc * dTdx;')]),
    ('v_mu_left', [('const double mu = 0.5 * (B->mu[bl] + B->mu[br]);',
      'const double mu = B->mu[bl];')]),
    ('v_kc_left', [('const double kc = 0.5 * (B->kc[bl] + B->kc[br]);',
      'const double kc = B->kc[bl];')]),
    ('v_cross2', [('/ (4.0 * P->dx[b]);',
      '/ (2.0 * P->dx[b]);')]),
    ('v_utau_left', [('utau += 0.5 * (bW(B, a, cl) + bW(B, a, cr)) * tau;',
      'utau += bW(B, a, cl) * tau;')]),
    ('g_energy0', [('S[1 + nd] += B.rho[b0] * B.W[(size_t)d * B.cnt + b0] * P->grav[d];',
      'S[1 + nd] += 0.0;')]),
    ('upd_sign', [('double R = S[v] - div;',
      'double R = S[v] + div;')]),
    ('capj_upd', [('R += (Gd[d][g * fc + fhi] + Gd[d][g * fc + flo]) / P->dx[d];',
      'R += (Gd[d][g * fc + fhi] - Gd[d][g * fc + flo]) / P->dx[d];')]),
    ('lsrk_swap', [('{0.25, 1.0 / 3.0, 0.5, 1.0}',
      '{1.0 / 3.0, 0.25, 0.5, 1.0}')]),
    ('thinc_F', [('F = (x3 - mn + gam) / (mx - mn + gam);',
      'F = (x3 - mn + gam) / (mx + gam);')]),
    ('muscl_R', [('if (dr != 0.0) *R = x3 - 0.5 * or_limiter(id, dc / dr) * dr;',
      'if (dr != 0.0) *R = x3 - 0.5 * or_limiter(id, dr / dc) * dr;')]),
    ('sg_e_pinf', [('return (p + c->gamma * c->pinf) / ((c->gamma - 1.0) * rho_k) + c->q;',
      'return (p + c->pinf) / ((c->gamma - 1.0) * rho_k) + c->q;')]),
    ('sg_inv_den', [('den += Y[k] * c->cv * (p + c->gamma * c->pinf) / (p + c->pinf);',
      'den += Y[k] * c->cv;')]),
    ('dt_state_end', [('*dt = cfl / smax;',
      '*dt = cfl / smax * 1.001;')]),
    ('lim_koren_orient', [('(1.0 + 2.0 * r) / 3.0',
      '(2.0 + r) / 3.0')]),
    ('lim_chak', [('fmin(1.0, 4.0 * r)',
      'fmin(1.0, 2.0 * r)')]),
    ('lim_vanalbada', [('(r + r * r) / (1.0 + r * r)',
      '(r + r * r) / (1.0 + r)')]),
    ('thinc_E', [('/ cosh(beta) - 1.0) / tanh(beta)',
      '/ sinh(beta) - 1.0) / tanh(beta)')]),
    ('thinc_mn', [('double mn = fmin(x1, x3), mx = fmax(x1, x3);',
      'double mn = fmin(x1, x2), mx = fmax(x1, x3);')]),
    ('baro_c2M', [('return p >= c->psat ? c->cl * c->cl : c->psat / c->rho_sl;',
      'return p >= c->psat ? c->cl * c->cl : c->psat / c->rho_sv;')]),
    ('baro_cap', [('if (s > 0.995) s = 0.995;',
      'if (s > 0.999) s = 0.999;')]),
    ('baro_snd_gas', [('inv += a / p;                          /* rho_i c_i^2',
      'inv += a / (1.4 * p);                          /* rho_i c_i^2')]),
    ('baro_snd_branch', [('const double c2 = rlm >= cl->rho_sl ? cl->cl * cl->cl : cl->psat / cl->rho_sl;',
      'const double c2 = rlm >= cl->rho_sl ? cl->psat / cl->rho_sl : cl->cl * cl->cl;')]),
    ('baro_gas_rho', [('return p / c->rt;                                                          /* Eq. 2-5 */',
      'return p / (1.01 * c->rt);')]),
    ('pr_first_root', [('                if (g < gbest) { gbest = g; best = Z; }',
      '                if (gbest == INFINITY) { gbest = g; best = Z; }')]),
    ('pr_c_isothermal', [('const double c2 = dpdrho + T * dpdT * dpdT / (rho * rho * pr_cv(m, T, v));',
      'const double c2 = dpdrho;')]),
    ('pr_cv_sign', [('return m->cvig - T * m->d2a',
      'return m->cvig + T * m->d2a')]),
    ('pr_d2a', [('A * cc * cc / (2.0 * T * Tc)',
      'A * cc * cc / (4.0 * T * Tc)')]),
    ('pr_b_coef', [('m->b += m->X[k] * 0.077796 * PR_RU',
      'm->b += m->X[k] * 0.0778 * 1.01 * PR_RU')]),
    ('in_u_index', [('w[a] = P->in_u ? P->in_u[a * fn + fc] : P->in_u0[a];',
      'w[a] = P->in_u ? P->in_u[fc] : P->in_u0[a];')]),
    ('sens_vap_thr', [('a5[2] > P->thr_vap',
      'a5[2] > 2.0 * P->thr_vap')]),
    ('sens_tv_onesided', [('tv += fabs(B->av[b0] - B->av[bm]) + fabs(B->av[bp] - B->av[b0]);',
      'tv += fabs(B->av[bp] - B->av[b0]);')]),
    ('hf_3cell', [('for (int m = -2; m <= 2; ++m) {',
      'for (int m = -1; m <= 1; ++m) {')]),
    ('hf_H_scale', [('h += B->al[bidx(B, q[0], q[1], q[2])] * P->dx[dir];',
      'h += B->al[bidx(B, q[0], q[1], q[2])];')]),
    ('csf_galpha_avg', [('galpha[d] += gu[d] / nvtx;',
      'galpha[d] += gu[d] / (nvtx - 1);')]),
    ('clip_tracked', [('Y[k] = clip01(Yt[k]);',
      'Y[k] = Yt[k];')]),
    ('clip_last', [('Y[N - 1] = clip01(1.0 - s);',
      'Y[N - 1] = 1.0 - s;')]),
    ('lsrk_a4', [('{0.25, 1.0 / 3.0, 0.5, 1.0}',
      '{0.25, 1.0 / 3.0, 0.5, 0.9}')]),
    ('grav_dir0', [('S[1 + d] += B.rho[b0] * P->grav[d];',
      'S[1 + d] += B.rho[b0] * P->grav[0];')]),
    ('vapour_alpha', [('return alpha[P->liquid] * s;',
      'return s;')]),
    ('baro_thinc_rho_mono', [('rho_monotone(rho4[1], rho4[2], rho4[3]) &&',
      '1 &&')]),
    ('sens_gas_liquidfrac', [('double ag0 = 1.0 - B->al[b0];',
      'double ag0 = B->al[b0];')]),
    ('bc_out_hi', [('    default: return n - 1;\n    }\n}',
      '    default: return n - 2 < 0 ? 0 : n - 2;\n    }\n}')]),
    ('in_disc_centre', [('double y = (src[1] + 0.5) * P->dx[1]',
      'double y = (src[1] + 0.0) * P->dx[1]')]),
    ('smooth_3d_weight', [('double wt = w3[a + 1] * (ry ? w3[b + 1] : 1.0) * (rz ? w3[c + 1] : 1.0);',
      'double wt = w3[a + 1] * (ry ? w3[b + 1] : 1.0);')]),
    ('step_qprev_q0', [('if ((st = or_stage(P, 3, dt, q0, qb, qa, NULL, NULL))) goto out;',
      'if ((st = or_stage(P, 3, dt, q0, q0, qa, NULL, NULL))) goto out;')]),
    ('step_base_qa', [('if ((st = or_stage(P, 2, dt, q0, qa, qb, NULL, NULL))) goto out;',
      'if ((st = or_stage(P, 2, dt, qa, qa, qb, NULL, NULL))) goto out;')]),
    ('slip_noflip', [('flip[0] = 1;   /* slip wall */',
      'flip[0] = 0;   /* slip wall */')]),
    ('capj_ghost_kap', [('                        kl = kap[mapped_cell(P, c)];',
      '                        kl = kap[mapped_cell(P, cp)];')]),
    ('hf_3d_Hy', [('const double Hy = (H[1][2] - H[1][0]) / (2.0 * d2);',
      'const double Hy = (H[1][2] - H[1][0]) / (2.0 * d1);')]),
    ('hf_3d_Hxy', [('(4.0 * d1 * d2)',
      '(2.0 * d1 * d2)')]),
    ('v_3d_dz', [('lp[b] += 1; lm[b] -= 1; rp[b] += 1; rm[b] -= 1;',
      'lp[b] += 1; lm[b] -= 1; rp[b] += 1; rm[b] -= (b == 2 ? 0 : 1);')]),
    ('csf_kappa_scale', [('kappa -= sg * nrm[d] / (scale * P->dx[d]);',
      'kappa -= sg * nrm[d] / (scale * P->dx[0]);')]),
    ('csf_vertex_off', [('c3[d] = (d < nd) ? ijk[d] + voff[d] - 1 + b[d] : ijk[d];',
      'c3[d] = (d < nd) ? ijk[d] + voff[d] + b[d] - (d == 1 ? 0 : 1) : ijk[d];')]),
    ('sens_dx', [('/ (2.0 * P->dx[bd]);\n        tg +=',
      '/ (2.0 * P->dx[0]);\n        tg +=')]),
    ('grad_eps_dxmax', [('for (int d = 1; d < nd; ++d) dxmin = fmin(dxmin, P->dx[d]);',
      'for (int d = 1; d < nd; ++d) dxmin = fmax(dxmin, P->dx[d]);')]),
    ('pr_e_dep_sign', [('return m->cvig * T + (m->a - T * m->da)',
      'return m->cvig * T + (m->a + T * m->da)')]),
    ('pr_inv_T', [('if (pr_e(&m, mid, v) > e) hi = mid; else lo = mid;',
      'if (pr_e(&m, mid, v) > e * 1.000001) hi = mid; else lo = mid;')]),
    ('baro_inv', [('if (bar_G(P, Y, v, mid) > 0.0) lo = mid; else hi = mid;',
      'if (bar_G(P, Y, v, mid) > 1e-9 * v) lo = mid; else hi = mid;')]),
    ('d3_scale_fixed', [('double d3 = P->d3p_coef * (',
      'double d3 = 0.5 * (')]),
    ('smooth_J', [('us = uL - (d3 - J) / (IL + IR);',
      'us = uL - (d3 + J) / (IL + IR);')]),
    ('totals_plain', [('if (fabs(s) >= fabs(x)) comp += (s - t) + x; else comp += (x - t) + s;',
      'comp += 0.0;')]),
    ('sg_inv_q', [('eq -= Y[k] * P->comp[k].q;',
      'eq -= 0.0 * P->comp[k].q;')]),
    ('sg_e_q', [('/ ((c->gamma - 1.0) * rho_k) + c->q;',
      '/ ((c->gamma - 1.0) * rho_k);')]),
    ('mix_kc_mu', [('k += al[c] * P->comp[c].kc;',
      'k += al[c] * P->comp[c].mu;')]),
    ('dt_max_not_sum', [('s += (fabs(w[d]) + cs) / P->dx[d];',
      's = fmax(s, (fabs(w[d]) + cs) / P->dx[d]);')]),
    ('dt_no_abs', [('s += (fabs(w[d]) + cs) / P->dx[d];',
      's += (w[d] + cs) / P->dx[d];')]),
    ('dt_dx_swapped', [('s += (fabs(w[d]) + cs) / P->dx[d];',
      's += (fabs(w[d]) + cs) / P->dx[nd - 1 - d];')]),
    ('dt_no_4_3', [('fmax(4.0 / 3.0 * mu, kc / cvmin)',
      'fmax(mu, kc / cvmin)')]),
    ('dt_no_2', [('s += 2.0 * fmax(',
      's += fmax(')]),
    ('dt_cv0', [('for (int k = 1; k < P->ncomp; ++k) cvmin = fmin(cvmin, P->comp[k].cv);',
      '')]),
    ('wood_mass_weighted', [('if (a > 0.0) inv += a / (P->comp[k].gamma * (p + P->comp[k].pinf));',
      'if (a > 0.0) inv += Y[k] / (P->comp[k].gamma * (p + P->comp[k].pinf));')]),
    ('rho_mass_weighted', [('v += Y[k] / rk[k];                                  /* Table A.1 density */', 'v += Y[k] * rk[k];'),
      ('    double r = 1.0 / v;\n    /* Eq. A.1.4', '    double r = v;\n    /* Eq. A.1.4')]),
    ('elig_no_eps_lo', [('return (x > eps) && (x < 1.0 - eps)',
      'return (x > 0.0) && (x < 1.0 - eps)')]),
    ('elig_no_eps_hi', [('return (x > eps) && (x < 1.0 - eps)',
      'return (x > eps) && (x < 1.0)')]),
    ('elig_no_monotone', [('&& ((x - xm) * (xp - x) > 0.0)',
      '')]),
    ('elig_L_cells', [('if (thinc_eligible(P->thinc_eps, w1[v], w2[v], w3[v])) WL[v] = tl;',
      'if (thinc_eligible(P->thinc_eps, w2[v], w3[v], w4[v])) WL[v] = tl;')]),
    ('elig_R_cells', [('if (thinc_eligible(P->thinc_eps, w2[v], w3[v], w4[v])) WR[v] = tr;',
      'if (thinc_eligible(P->thinc_eps, w1[v], w2[v], w3[v])) WR[v] = tr;')]),
    ('pr_X_is_Y', [('m->X[k] = (Y[k] / P->comp[k].M) * m->M;',
      'm->X[k] = Y[k];')]),
    ('pr_Tc_i', [('double Tc = sqrt(ci->Tc * cj->Tc);',
      'double Tc = ci->Tc;')]),
    ('pr_Tc_mean', [('double Tc = sqrt(ci->Tc * cj->Tc);',
      'double Tc = 0.5 * (ci->Tc + cj->Tc);')]),
    ('pr_vc_mean', [('double vc = pow(cbrt(vci) + cbrt(vcj), 3.0) / 8.0;',
      'double vc = 0.5 * (vci + vcj);')]),
    ('pr_w_i', [('double w = 0.5 * (ci->omega + cj->omega);',
      'double w = ci->omega;')]),
    ('muscl_L_ratio', [('if (dl != 0.0) *L = x2 + 0.5 * or_limiter(id, dc / dl) * dl;',
      'if (dl != 0.0) *L = x2 + 0.5 * or_limiter(id, dl / dc) * dl;')]),
    ('koren_cap', [('case OR_KOREN: return fmax(0.0, min3(2.0, 2.0 * r,',
      'case OR_KOREN: return fmax(0.0, min3(1.5, 2.0 * r,')]),
    ('thinc_E_arg', [('exp(theta * beta * (2.0 * F - 1.0))',
      'exp(theta * beta * (F - 0.5))')]),
    ('pr_gdep_sign', [('return Z - 1.0 - log(Z - B) - A / (2.0 * s2 * B)',
      'return Z - 1.0 - log(Z - B) + A / (2.0 * s2 * B)')]),
    ('pr_dpdrho', [('const double dpdrho = -(v * v / m->M) * dpdv;',
      'const double dpdrho = -(v / m->M) * dpdv;')]),
    ('baro_wood', [('if (a > 0.0) inv += a / (rk[k] * bar_c2_k(&P->comp[k], p));',
      'if (a > 0.0) inv += a / bar_c2_k(&P->comp[k], p);')]),
    ('vapour_denom', [('double s = (c->rho_sl - rlm) / (c->rho_sl - c->rho_sv);',
      'double s = (c->rho_sl - rlm) / c->rho_sl;')]),
    ('visc_normal_2dx', [('g[a][b] = (bW(B, a, cr) - bW(B, a, cl)) / P->dx[d];',
      'g[a][b] = (bW(B, a, cr) - bW(B, a, cl)) / (2.0 * P->dx[d]);')]),
    ('visc_dT_dx0', [('const double dTdx = (bW(B, nd + 1, cr) - bW(B, nd + 1, cl)) / P->dx[d];',
      'const double dTdx = (bW(B, nd + 1, cr) - bW(B, nd + 1, cl)) / P->dx[0];')]),
    ('grav_energy_u0', [('S[1 + nd] += B.rho[b0] * B.W[(size_t)d * B.cnt + b0] * P->grav[d];',
      'S[1 + nd] += B.rho[b0] * B.W[0] * P->grav[d];')]),
    ('inflow_src1', [('                        src[0] = 0;\n                        flip[0] = 0;',
      '                        src[0] = 1;\n                        flip[0] = 0;')]),
    ('inflow_dz_yc', [('double dy = y - P->in_yc, dz = (nd == 3) ? z - P->in_zc : 0.0;',
      'double dy = y - P->in_yc, dz = (nd == 3) ? z - P->in_yc : 0.0;')]),
    ('step_time2', [('if (t) *t += dt;',
      'if (t) *t += 2.0 * dt;')]),
    ('cp_Y_unscaled', [('for (int k = 0; k < N - 1; ++k) Yt[k] = qc[2 + nd + k] / rho;',
      'for (int k = 0; k < N - 1; ++k) Yt[k] = qc[2 + nd + k];')]),
    ('p2c_energy', [('q[(size_t)(1 + nd) * nc + c] = r * (e + ke);',
      'q[(size_t)(1 + nd) * nc + c] = r * e + ke;')]),
    ('hf_Hx_1dx', [('const double Hx = (H[2][1] - H[0][1]) / (2.0 * d1);',
      'const double Hx = (H[2][1] - H[0][1]) / d1;')]),
    ('csf_energy_sign', [('S[nd] = P->sigma * kappa * udg;',
      'S[nd] = -P->sigma * kappa * udg;')]),
    ('baro_e_fourth', [('const int fourth = (v < iY) && !(baro && v == iT);',
      'const int fourth = (v < iY);')]),
    ('sens_thr_gas', [('a5[1] > P->thr_gas',
      'a5[1] > 2.0 * P->thr_gas')]),
    ('sens_eps_ducros', [('a5[0] = div * div / (div * div + curl2 + P->eps_ducros);',
      'a5[0] = div * div / (div * div + curl2 + 1e-6);')]),
    ('capj_energy_g', [('const int g = (v == 1 + nd) ? 1 : 0;',
      'const int g = 0;')]),
    ('smooth_norm', [('return s / norm;   /* norm = 16 in 2D, 64 in 3D */',
      'return s / 16.0;')]),
    ('mix_mu_first', [('m += al[c] * P->comp[c].mu;',
      'm += al[0] * P->comp[c].mu;')]),
    ('p2c_species_idx', [('q[(size_t)(2 + nd + k) * nc + c] = r * w[nd + 2 + k];',
      'q[(size_t)(2 + nd + k) * nc + c] = r * w[nd + 2];')]),
    ('cp_species_idx', [('for (int k = 0; k < N - 1; ++k) Yt[k] = qc[2 + nd + k] / rho;',
      'for (int k = 0; k < N - 1; ++k) Yt[k] = qc[2 + nd] / rho;')]),
    ('flux_species_idx', [('for (int k = 0; k < N - 1; ++k) F[2 + nd + k] = us * rs * Ws[iY + k];',
      'for (int k = 0; k < N - 1; ++k) F[2 + nd + k] = us * rs * Ws[iY];')]),
    ('inflow_Y_idx', [('for (int kk = 0; kk < P->ncomp - 1; ++kk) w[nd + 2 + kk] = P->in_Y[kk];',
      'for (int kk = 0; kk < P->ncomp - 1; ++kk) w[nd + 2 + kk] = P->in_Y[0];')]),
    ('visc_mom_idx', [('        F[1 + a] -= tau;',
      '        F[1 + d] -= tau;')]),
    ('csf_force_idx', [('S[d] = P->sigma * kappa * galpha[d];',
      'S[d] = P->sigma * kappa * galpha[0];')]),
    ('hf_swap_ab', [('                q[t[0]] += a;\n                if (nt == 2) q[t[1]] += b;',
      '                q[t[0]] += b;\n                if (nt == 2) q[t[1]] += a;')]),
    ('mom_flux_u_idx', [('for (int a = 0; a < nd; ++a) F[1 + a] = us * rs * Ws[a] + (a == d ? ps : 0.0);',
      'for (int a = 0; a < nd; ++a) F[1 + a] = us * rs * Ws[d] + (a == d ? ps : 0.0);')]),
    ('sg_alpha_idx', [('double a = (Y[k] > 0.0) ? r * Y[k] / rk[k] : 0.0;\n        if (alpha) alpha[k] = a;\n        if (a > 0.0) inv += a / (P->comp[k].gamma',
      'double a = (Y[k] > 0.0) ? r * Y[k] / rk[0] : 0.0;\n        if (alpha) alpha[k] = a;\n        if (a > 0.0) inv += a / (P->comp[k].gamma')]),
    ('liquid_index_fixed', [('B->al[b] = alk[P->liquid];',
      'B->al[b] = alk[1];')]),
    ('baro_vapour_liquid_idx', [('    const or_comp* c = &P->comp[P->liquid];\n    const double rlm = bar_rho_k(c, p);',
      '    const or_comp* c = &P->comp[1];\n    const double rlm = bar_rho_k(c, p);')]),
    ('baro_snd_liquid_idx', [('const int N = P->ncomp, L = P->liquid;',
      'const int N = P->ncomp, L = 1;')]),
    ('baro_vapour_alpha_idx', [('return alpha[P->liquid] * s;',
      'return alpha[1] * s;')]),
    ('param_beta', [('or_thinc(P->beta, P->thinc_gamma, w1[v], w2[v], w3[v], w4[v], &tl, &tr);',
      'or_thinc(1.6, P->thinc_gamma, w1[v], w2[v], w3[v], w4[v], &tl, &tr);')]),
    ('param_thinc_eps', [('if (thinc_eligible(P->thinc_eps, w1[v], w2[v], w3[v])) WL[v] = tl;',
      'if (thinc_eligible(1e-4, w1[v], w2[v], w3[v])) WL[v] = tl;')]),
    ('param_limiters', [('int lim = (v < nd) ? P->lim_vel : P->lim_scalar;',
      'int lim = (v < nd) ? OR_KOREN : OR_MINMOD;')]),
    ('param_thr_ducros', [('(a5[0] > P->thr_ducros ||',
      '(a5[0] > 0.95 ||')]),
    ('param_eps_ducros', [('a5[0] = div * div / (div * div + curl2 + P->eps_ducros);',
      'a5[0] = div * div / (div * div + curl2 + 1e-20);')]),
    ('param_grad_eps', [('if (mag > P->grad_eps / dxmin)',
      'if (mag > 1e-5 / dxmin)')]),
]


def pins():
    """the CPU pins of the oracle (never this check's own sampled test)"""
    tests = sorted(os.path.join("tests", f) for f in os.listdir(os.path.join(ROOT, "tests"))
                   if f.startswith("test_oracle_") and f.endswith(".py"))
    return tests + [os.path.join("tests", "test_workloads.py")]


def run_one(src, name, pairs, tests):
    """(name, caught, first failing test)"""
    text = src
    for old, new in pairs:
        if text.count(old) != 1:
            raise ValueError(f"{name}: the planted text occurs {text.count(old)} times")
        text = text.replace(old, new)
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        shutil.copytree(HERE, os.path.join(d, "oracle"),
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
        with open(os.path.join(d, "oracle", "oracle.c"), "w") as f:
            f.write(text)
        code = ("import sys; sys.path.insert(0, %r); import oracle; assert oracle.__file__.startswith(%r); "
                "import pytest; sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider'] + %r))" % (d, d, tests))
        env = dict(os.environ, OMP_NUM_THREADS="2")
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, env=env)
        failed = [l for l in r.stdout.splitlines() if l.startswith("FAILED")][:1]
        if r.returncode not in (0, 1):
            raise RuntimeError(f"{name}: pytest exited {r.returncode}\n{r.stdout[-2000:]}{r.stderr[-2000:]}")
        return name, r.returncode == 1, failed[0][7:] if failed else ""
    finally:
        shutil.rmtree(d, ignore_errors=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("-j", type=int, default=4, help="mistakes checked at once")
    ap.add_argument("names", nargs="*")
    a = ap.parse_args()
    src = open(os.path.join(HERE, "oracle.c")).read()
    todo = [m for m in MUTANTS if not a.names or m[0] in a.names]
    tests = pins()
    missed = []
    with ThreadPoolExecutor(a.j) as ex:
        for name, caught, first in ex.map(lambda m: run_one(src, m[0], m[1], tests), todo):
            print(f"{name:24s} {'caught by ' + first if caught else 'NOT CAUGHT'}", flush=True)
            if not caught:
                missed.append(name)
    unexpected = sorted(set(missed) - ACCEPTED)
    print(f"{len(todo)} planted, {len(todo) - len(missed)} caught; not caught: {sorted(missed)}")
    sys.exit(1 if unexpected else 0)


if __name__ == "__main__":
    main()
