"""The oracle's pins catch plausible mistakes anywhere in the oracle: each of
the 61 mutants below plants one (a dropped term, a wrong sign, factor or
index, a transposed operand, a wrong constant) in a copy of the oracle's C
source, is built, and must fail at least one pin (the Monte-Carlo estimate with the
rich prior aside, for time).  The mutants cover every function the CUDA path
is compared with: Q(beta) (Eq. 19-21, 27), the sums (Eq. 17, 24, 25),
Q(rho) and Q(K, Lambda) (Eq. 16-18, 22-25), every ELBO term, the Wishart and
digamma helpers, the linear algebra, the profile-grouped sums and fit, the
stopping tests, the ELBO of given factors and EM (Eq. 42-47).  (Dropping the
explicit symmetrisation of EM's Lambda^{-1} is not among them: the matrix is
symmetric before it up to the last bit, so that mutant is equivalent.)"""
import concurrent.futures as cf
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC_PATH = os.path.join(ROOT, "oracle", "vbh_oracle.c")

MUTANTS = [  # name, text, replacement, which occurrence (0-based)
 ("eq20_drop_rho", "Lb[j * M + k] = EL[j * M + k] + Erho * D[j] * D[k];   /* Eq. 20 */", "Lb[j * M + k] = EL[j * M + k];   /* Eq. 20 */", 0),
 ("eq21_rhs_half", "rhs[j] = ELK[j] + Erho * D[j] * yt;", "rhs[j] = ELK[j] + 0.5 * Erho * D[j] * yt;", 0),
 ("eq31_index", "t += EL[j * M + k] * g->kappa[k];", "t += EL[j * M + k] * g->kappa[j];", 0),
 ("eq17_sign", "s->sum_S += yt * yt - 2.0 * yt * Dmu + DEbbD;", "s->sum_S += yt * yt + 2.0 * yt * Dmu + DEbbD;", 0),
 ("eq27_drop_sigma", "Ebb[j * M + k] = mi[j] * mi[k] + Si[j * M + k];", "Ebb[j * M + k] = mi[j] * mi[k];", 0),
 ("eq16_b_factor", "g->b_rho = p->b0 + 0.5 * s->sum_S;", "g->b_rho = p->b0 + s->sum_S;", 0),
 ("eq16_a_factor", "g->a_rho = p->a0 + 0.5 * s->V;", "g->a_rho = p->a0 + s->V;", 0),
 ("eq22_lam", "g->lam = p->q0 + V;", "g->lam = V;", 0),
 ("eq22_nu", "g->nu = p->n0 + V;", "g->nu = p->n0 + V + 1.0;", 0),
 ("eq24_drop_prior", "(s->sum_mu[j] + p->q0 * p->K0[j]) / (V + p->q0)", "(s->sum_mu[j]) / (V + p->q0)", 0),
 ("eq25_K0_index", "+ p->q0 * p->K0[j] * p->K0[k]", "+ p->q0 * p->K0[j] * p->K0[j]", 0),
 ("eq25_Ebb_index", "p->L0inv[j * M + k] + s->sum_Ebb[j * M + k]", "p->L0inv[j * M + k] + s->sum_Ebb[j * M + j]", 0),
 ("eq25_drop_L0", "g->Winv[j * M + k] = p->L0inv[j * M + k] + s->sum_Ebb", "g->Winv[j * M + k] = s->sum_Ebb", 0),
 ("elbo_lik_sign", "- 0.5 * Erho * s->sum_S;", "+ 0.5 * Erho * s->sum_S;", 0),
 ("elbo_beta_drop_lam", " - 0.5 * V * M / g->lam;", ";", 0),
 ("elbo_K_drop_lam", "- 0.5 * p->q0 * (quadK + M / g->lam);", "- 0.5 * p->q0 * quadK;", 0),
 ("elbo_quadK_index", "(g->kappa[k] - p->K0[k]);", "(g->kappa[k] - p->K0[j]);", 0),
 ("elbo_C_sign", "- s->sum_mu[j] * g->kappa[k] + V * g->kappa[j] * g->kappa[k];", "+ s->sum_mu[j] * g->kappa[k] + V * g->kappa[j] * g->kappa[k];", 0),
 ("elbo_hbeta_const", "0.5 * V * M * (1.0 + VBO_LN2PI)", "0.5 * V * M * VBO_LN2PI", 0),
 ("elbo_hK_sign", "(log(g->lam) - VBO_LN2PI) + 0.5 * M;", "(log(g->lam) - VBO_LN2PI) - 0.5 * M;", 0),
 ("elbo_hrho_sign", "(1.0 - g->a_rho) * vbo_digamma(g->a_rho)", "(1.0 + g->a_rho) * vbo_digamma(g->a_rho)", 0),
 ("elbo_trho", "(p->a0 - 1.0) * Elnrho", "(p->a0 + 1.0) * Elnrho", 0),
 ("elbo_tLam", "0.5 * (p->n0 - M - 1.0) * ElnL", "0.5 * (p->n0 - M) * ElnL", 0),
 ("elbo_trL0_drop", "- 0.5 * trL0EL;", ";", 0),
 ("elbo_hLam_nuM", "+ 0.5 * g->nu * M)", ")", 0),
 ("wishart_Elndet_ln2", "double s = M * VBO_LN2 + lndetW;", "double s = lndetW;", 0),
 ("wishart_lnB_pi", "0.25 * M * (M - 1) * VBO_LNPI", "0.25 * M * M * VBO_LNPI", 0),
 ("wishart_lnB_lgamma", "s -= lgamma(0.5 * (nu + 1.0 - j));", "s -= lgamma(0.5 * (nu - j));", 0),
 ("digamma_series", "1.0 / 252.0", "1.0 / 250.0", 0),
 ("digamma_recurrence", "acc -= 1.0 / x;", "acc -= 1.0 / (x + 1.0);", 0),
 ("observation_mu", "*yt = (double)r[i] - dS;", "*yt = (double)r[i];", 0),
 ("observation_D", "D[j] = (double)d[i * S + j] - dS;", "D[j] = (double)d[i * S + j];", 0),
 ("beta_init_half", "Sig[i * M * M + j] = p->L0inv[j];", "Sig[i * M * M + j] = 0.5 * p->L0inv[j];", 0),
 ("grouped_sumS", "s->sum_S += y2 - 2.0 * (Da * y1 + Db * y2) + DEbbD;", "s->sum_S += y2 - 2.0 * (Da * y1 + Db * y1) + DEbbD;", 0),
 ("grouped_Ebb", "+ b[j] * b[k] * y2;", "+ b[j] * b[k] * y1;", 0),
 ("grouped_logdet", "s->sum_logdet += nq * ld;", "s->sum_logdet += ld;", 0),
 ("grouped_b", "b[j] = Erho * tb;", "b[j] = tb;", 0),
 ("em_rho", "out->rho = Vd / sumS;", "out->rho = (Vd - 1.0) / sumS;", 0),
 ("em_Linv_drop_KK", "sumMM[j * M + k] / Vd - out->K[j] * out->K[k]", "sumMM[j * M + k] / Vd", 0),
 ("em_loglik_var_index", "var += D[j] * t->Linv[j * M + k] * D[k];", "var += D[j] * t->Linv[j * M + k] * D[j];", 0),
 ("em_DQD_drop_sig", "DQD += D[j] * (Mi[j] * Mi[k] + Sig[j * M + k]) * D[k];", "DQD += D[j] * (Mi[j] * Mi[k]) * D[k];", 0),
 ("em_loglik_log", "log(var) + e * e / var", "e * e / var", 0),
 ("chol_transposed", "s -= L[j * M + k] * L[j * M + k];", "s -= L[j * M + k] * L[k * M + j];", 0),
 ("inverse_back_transposed", "t -= L[k * M + i] * x[k];", "t -= L[i * M + k] * x[k];", 0),
 ("logdet_half", "s += 2.0 * log(L[j * M + j]);", "s += log(L[j * M + j]);", 1),
 ("inverse_logdet_half", "s += 2.0 * log(L[j * M + j]);", "s += log(L[j * M + j]);", 0),
 ("fit_tol_absolute", "if (fabs(L - Lprev) < tol * fabs(L))", "if (fabs(L - Lprev) < tol)", 0),
    ("elbo_at_init_beta", "if (vbo_beta_update(p, V, r, d, g, mu, Sig)) { rc = -1; goto done; }\n    if (vbo_sums_from_beta(p, V, r, d, mu, Sig, &s)) { rc = -1; goto done; }\n    if (vbo_elbo(p, &s, g, elbo, const_dropped)) rc = -1;",
     "vbo_beta_init(p, V, mu, Sig);\n    if (vbo_sums_from_beta(p, V, r, d, mu, Sig, &s)) { rc = -1; goto done; }\n    if (vbo_elbo(p, &s, g, elbo, const_dropped)) rc = -1;", 0),
    ("grouped_fit_tol_abs", "if (fabs(L - Lprev) < tol * fabs(L)) { *converged = 1; break; }", "if (fabs(L - Lprev) < tol) { *converged = 1; break; }", 1),
    ("em_fit_iters", "*iters = n;", "*iters = n + 1;", 0),
    ("em_loglik_mean_index", "mean += D[j] * t->K[j];", "mean += D[j] * t->K[0];", 0),
    ("beta_Erho_mode", "double Erho = g->a_rho / g->b_rho;", "double Erho = (g->a_rho - 1.0) / g->b_rho;", 0),
    ("elbo_Erho_mode", "double Erho = g->a_rho / g->b_rho;", "double Erho = (g->a_rho - 1.0) / g->b_rho;", 1),
    ("elbo_Elnrho_log", "vbo_digamma(g->a_rho) - log(g->b_rho)", "log(g->a_rho) - log(g->b_rho)", 0),
    ("beta_EL_unscaled", "EL[j] *= g->nu;", "EL[j] *= 1.0;", 0),
    ("grouped_EL_unscaled", "EL[j] *= g->nu;", "EL[j] *= 1.0;", 1),
    ("elbo_EL_unscaled", "EL[j] *= g->nu;", "EL[j] *= 1.0;", 2),
    ("grouped_mus_y2", "mus[j] = nq * a[j] + b[j] * y1;", "mus[j] = nq * a[j] + b[j] * y2;", 0),
    ("grouped_Sg_count", "Ebb[j * M + k] = nq * Sg[j * M + k]", "Ebb[j * M + k] = Sg[j * M + k]", 0),
    ("sums_V_offbyone", "s->V = (double)V;", "s->V = (double)V + 1.0;", 0),
    ("grouped_erho_inverted", "Erho = g->a_rho / g->b_rho;\n    }", "Erho = g->b_rho / g->a_rho;\n    }", 0),
]


def _mutant_source(src, text, replacement, occ):
    idx, start = -1, 0
    for _ in range(occ + 1):
        idx = src.find(text, start)
        assert idx >= 0, text
        start = idx + 1
    return src[:idx] + replacement + src[idx + len(text):]


def _killed(src, odir, m):
    name, text, replacement, occ = m
    c, so = os.path.join(odir, name + ".c"), os.path.join(odir, name + ".so")
    with open(c, "w") as f:
        f.write(_mutant_source(src, text, replacement, occ))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", c, "-lm", "-o", so])
    code = ("import sys\n"
            f"sys.path.insert(0, {ROOT!r})\n"
            "import oracle.oracle as O\n"
            f"O._LIB = {so!r}\n"
            "O.build = lambda force=False: O._LIB\n"
            "import pytest\n"
            "sys.exit(int(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', '-k', 'not monte_carlo',\n"
            f"    {os.path.join(ROOT, 'tests', 'test_oracle_pins.py')!r},\n"
            f"    {os.path.join(ROOT, 'tests', 'test_oracle_em_pins.py')!r}])))\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900)
    return name, out.returncode != 0


def test_every_mutant_of_the_oracle_fails_a_pin():
    with open(SRC_PATH) as f:
        src = f.read()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    odir = os.path.join(ROOT, "oracle", "_build", "mutants")
    os.makedirs(odir, exist_ok=True)
    with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        res = list(ex.map(lambda m: _killed(src, odir, m), MUTANTS))
    survivors = [n for n, k in res if not k]
    assert not survivors, survivors
