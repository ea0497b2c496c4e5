"""The oracle's pins against planted mistakes.

Each case copies ``oracle/``, ``synth/`` and ``tests/`` to a temporary
directory, plants one plausible mistake in the copied oracle (a dropped term,
a wrong sign, index or scale, a transposed or mirrored operand) and runs the
oracle's pin tests there: at least one pin must fail on an assertion.  The
mistakes live only in the temporary copy; nothing here touches the GPU path.
Tests that restate a formula (the FDK filter against its own convolution sum)
are left out, since a restatement cannot catch its own mistake.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FB = ["tests/test_oracle_fblisa.py", "tests/test_golden_paper.py"]
PROJ = ["tests/test_oracle_projector.py"]
FDK = ["tests/test_oracle_fdk.py"]
TV = ["tests/test_oracle_tv.py"]
MLP = ["tests/test_oracle_mlp.py"]
PROP = ["tests/test_oracle_proposal.py"]

# (oracle file, text, planted replacement, pin files)
MUTATIONS = {
    # Algorithm 1 (oracle/fblisa.py)
    "fb_grad_scale": ("fblisa.py", "    g = scale * backproject(geom, r, views)",
                      "    g = backproject(geom, r, views)", FB),
    "fb_f_scale": ("fblisa.py", "    f_x = 0.5 * scale * rho0", "    f_x = 0.5 * rho0", FB),
    "fb_fbar_scale": ("fblisa.py", "        f_xbar = 0.5 * scale * rho1", "        f_xbar = 0.5 * rho1", FB),
    "fb_rhs_half": ("fblisa.py", "rhs = f_x + gTd + dd / (2.0 * alpha)", "rhs = f_x + gTd + dd / alpha", FB),
    "fb_rhs_sign": ("fblisa.py", "rhs = f_x + gTd + dd / (2.0 * alpha)", "rhs = f_x - gTd + dd / (2.0 * alpha)", FB),
    "fb_prox_threshold": ("fblisa.py", "    return np.maximum(v - alpha * mu, 0.0)",
                          "    return np.maximum(v - mu, 0.0)", FB),
    "fb_fisher_yates": ("fblisa.py", "        j = i + int(math.floor(u * (n - i)))",
                        "        j = i + int(math.floor(u * (n - i - 1)))", FB),
    "fb_schedule": ("fblisa.py", "        K = k_hat + -(-n_theta // N_prev)", "        K = k_hat", FB),
    "fb_no_padding": ("fblisa.py", "            sl = sl + perm[:N_t - len(sl)]", "            sl = sl", FB),
    "fb_residual_sign": ("fblisa.py", "    r = project(geom, x, views) - bS", "    r = bS - project(geom, x, views)", FB),
    "fb_epoch_key": ("fblisa.py", "    state = (seed ^ ((epoch * EPOCH_KEY) & MASK64)) & MASK64",
                     "    state = (seed ^ epoch) & MASK64", FB),
    "fb_splitmix_constant": ("fblisa.py", "    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64",
                             "    z = ((z ^ (z >> 27)) * 0x94D049BB133111EA) & MASK64", FB),
    "fb_splitmix_shift": ("fblisa.py", "    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64",
                          "    z = ((z ^ (z >> 31)) * 0xBF58476D1CE4E5B9) & MASK64", FB),
    # projector (oracle/joseph.c)
    "proj_no_obliquity": ("joseph.c", "    return V[a] * len / fabs(d[a]);", "    return V[a];", PROJ),
    "proj_no_voxel_size": ("joseph.c", "    return V[a] * len / fabs(d[a]);", "    return len / fabs(d[a]);", PROJ),
    "proj_mirrored_u": ("joseph.c", "    P[0] = -off * c - u * sn;\n    P[1] = -off * sn + u * c;",
                        "    P[0] = -off * c + u * sn;\n    P[1] = -off * sn - u * c;", PROJ),
    "proj_row_shift": ("joseph.c", "    double w = ((double)iv - 0.5 * (double)(g->nv - 1)) * g->dv;",
                       "    double w = ((double)iv - 0.5 * (double)g->nv) * g->dv;", PROJ),
    "proj_column_shift": ("joseph.c", "    double u = ((double)iu - 0.5 * (double)(g->nu - 1)) * g->du;",
                          "    double u = ((double)iu - 0.5 * (double)g->nu) * g->du;", PROJ),
    "proj_bilinear_swap": ("joseph.c", "            wt[n] = (db ? fb : 1.0 - fb) * (dc ? fc : 1.0 - fc);",
                           "            wt[n] = (db ? 1.0 - fb : fb) * (dc ? fc : 1.0 - fc);", PROJ),
    "proj_plane_shift": ("joseph.c", "    double plane = ((double)m - 0.5 * (double)(N[a] - 1)) * V[a];",
                         "    double plane = ((double)m - 0.5 * (double)N[a]) * V[a];", PROJ),
    "proj_unweighted_adjoint": ("joseph.c", "                for (int q = 0; q < n; ++q) acc[idx[q]] += wt[q] * wy;",
                                "                for (int q = 0; q < n; ++q) acc[idx[q]] += wy;", PROJ),
    "proj_source_side": ("joseph.c", "    s[0] = g->sod * c;\n    s[1] = g->sod * sn;",
                         "    s[0] = -g->sod * c;\n    s[1] = -g->sod * sn;", PROJ),
    "proj_inplane_scale": ("joseph.c", "    double qb = (s[b] + t * d[b]) / V[b] + 0.5 * (double)(N[b] - 1);",
                           "    double qb = (s[b] + t * d[b]) + 0.5 * (double)(N[b] - 1);", PROJ),
    # FDK (oracle/fdk.py)
    "fdk_odd_tap_sign": ("fdk.py", "h[odd] = -1.0 / (math.pi ** 2 * k[odd] ** 2 * t * t)",
                         "h[odd] = 1.0 / (math.pi ** 2 * k[odd] ** 2 * t * t)", FDK),
    "fdk_no_cosine": ("fdk.py", "    W = geom.sod / np.sqrt(geom.sod ** 2 + a[None, :] ** 2 + b[:, None] ** 2)",
                      "    W = np.ones((geom.nv, geom.nu))", FDK),
    "fdk_uniform_dtheta": ("fdk.py", "    dth = view_weights(ang)", "    dth = np.full(len(ang), 2 * math.pi / len(ang))", FDK),
    "fdk_1_over_U": ("fdk.py", "/ (U * U)", "/ U", FDK),
    "fdk_nearest": ("fdk.py", "    tv = fv - iv0\n    tu = fu - iu0\n", "    tv = np.round(fv - iv0)\n    tu = np.round(fu - iu0)\n", FDK),
    "fdk_no_t": ("fdk.py", "        q[s] = t * np.fft.irfft(", "        q[s] = np.fft.irfft(", FDK),
    "fdk_no_half": ("fdk.py", "f += 0.5 * dth[s]", "f += dth[s]", FDK),
    "fdk_mirrored_u": ("fdk.py", "        fu = (eta / U) / (geom.du * m) + cu", "        fu = -(eta / U) / (geom.du * m) + cu", FDK),
    "fdk_row_without_U": ("fdk.py", "        fv = (z / U) / (geom.dv * m) + cv", "        fv = z / (geom.dv * m) + cv", FDK),
    # other regularisers (oracle/tv.py)
    "tv_adjoint_sign": ("tv.py", "out[tuple(own)] -= q[c][tuple(own)]", "out[tuple(own)] += q[c][tuple(own)]", TV),
    "tv_adjoint_drop": ("tv.py", "        out[tuple(up)] += q[c][tuple(own)]\n", "", TV),
    "tv_anisotropic_projection": ("tv.py", "    return q / np.maximum(nrm, 1.0)[None]", "    return np.clip(q, -1, 1)", TV),
    "tv_no_box": ("tv.py", "        return np.clip(v - lam * grad_adjoint(p), 0.0, x_max)",
                  "        return v - lam * grad_adjoint(p)", TV),
    "l1_box_threshold": ("tv.py", "    return np.clip(v - a * mu, 0.0, x_max)", "    return np.clip(v - mu, 0.0, x_max)", TV),
    # step-proposal network (oracle/mlp.py)
    "mlp_tanh_derivative_2": ("mlp.py", '    dz2 = np.outer(dy, w["W3"]) * (1.0 - h2 * h2)',
                              '    dz2 = np.outer(dy, w["W3"]) * (1.0 + h2 * h2)', MLP),
    "mlp_tanh_derivative_1": ("mlp.py", '    dz1 = (dz2 @ w["W2"]) * (1.0 - h1 * h1)',
                              '    dz1 = (dz2 @ w["W2"]) * (1.0 - h1)', MLP),
    "mlp_loss_mean": ("mlp.py", "    dy = (y - np.asarray(t, dtype=np.float64)) / n",
                      "    dy = (y - np.asarray(t, dtype=np.float64))", MLP),
    "adam_bias_m": ("mlp.py", "    m_hat = m / (1.0 - beta1 ** step)", "    m_hat = m", MLP),
    "adam_bias_v": ("mlp.py", "    v_hat = v / (1.0 - beta2 ** step)", "    v_hat = v", MLP),
    "adam_eps_inside": ("mlp.py", "lr * m_hat / (np.sqrt(v_hat) + eps)", "lr * m_hat / np.sqrt(v_hat + eps)", MLP),
    # learned step proposal (oracle/proposal.py)
    "prop_base_zero": ("proposal.py", "    base = st.j_prev if st.have_prev else 0", "    base = 0", PROP),
    "prop_no_half": ("proposal.py", "base + pred + 0.5 - margin", "base + pred - margin", PROP),
    "prop_grid_extra": ("proposal.py", "    for _ in range(j):\n        a *= beta",
                        "    for _ in range(j + 1):\n        a *= beta", PROP),
    "prop_curvature_no_2": ("proposal.py", "alpha0 * g2 / max(2.0 * f, 1e-300)", "alpha0 * g2 / max(f, 1e-300)", PROP),
    "prop_grad_ratio_no_sqrt": ("proposal.py", "        out[2] = 0.5 * math.log(", "        out[2] = math.log(", PROP),
    "prop_absolute_f": ("proposal.py", "        out[1] = math.log(max(f, 1e-300) / max(st.f_prev, 1e-300))",
                        "        out[1] = math.log(max(f, 1e-300))", PROP),
    "prop_dj_after_update": ("proposal.py", "    st.dj_prev = j_acc - st.j_prev\n    st.have_dj = st.have_prev\n    st.j_prev = j_acc",
                             "    st.j_prev = j_acc\n    st.dj_prev = j_acc - st.j_prev\n    st.have_dj = st.have_prev", PROP),
    "prop_no_k_count": ("proposal.py", "    st.have_prev = True\n    st.k += 1", "    st.have_prev = True", PROP),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    fname, text, planted, pins = MUTATIONS[name]
    ign = shutil.ignore_patterns("__pycache__", "_build", "*.so")
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d, ignore=ign)
    path = tmp_path / "oracle" / fname
    src = path.read_text()
    assert src.count(text) >= 1, "the oracle no longer contains the text this case mutates"
    path.write_text(src.replace(text, planted, 1))
    env = dict(os.environ, PYTHONPATH=str(tmp_path), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", *pins, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", "-k", "not direct_convolution"],
                       cwd=tmp_path, env=env, capture_output=True, text=True, timeout=600)
    tail = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr[-400:]
    assert r.returncode == 1, "no pin caught the planted mistake (%s): %s" % (name, tail)
    assert " failed" in tail and "error" not in tail, tail
