"""The oracle's pins reject plausible mistakes (no GPU).

Each case plants one error in a copy of ``oracle/oracle.cpp`` (a dropped term,
a flipped sign, a wrong index, a transposed rotation, a wrong quadrature
weight ...), builds it in a temporary directory, and runs the pin suites
against that build through ``CISCVX_ORACLE_LIB``.  The pins must fail for
every planted error; the real oracle must pass (the other test files).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")
PINS = ["tests/test_oracle_integrator.py", "tests/test_oracle_physics.py", "tests/test_oracle_vjp.py",
        "tests/test_oracle_node.py", "tests/test_oracle_cross.py", "tests/test_oracle_paper_dynamics.py",
        "tests/test_oracle_psi.py"]

MUTATIONS = [
    ("Psi pair (phi_n, lambda^c) takes gamma", "out[2 * i] = fischer_burmeister(d[4 * i], d[4 * i + 1], delta);",
     "out[2 * i] = fischer_burmeister(d[4 * i], d[4 * i + 2], delta);"),
    ("Psi pair (gamma, rho^c) takes lambda^c", "out[2 * i + 1] = fischer_burmeister(d[4 * i + 2], d[4 * i + 3], delta);",
     "out[2 * i + 1] = fischer_burmeister(d[4 * i + 1], d[4 * i + 3], delta);"),
    ("Psi increment reversed", "d[j] = ym - yp;", "d[j] = yp - ym;"),
    ("Psi epsilon sign", "out[2 * nc + i] = d[4 * nc + i] - eps;", "out[2 * nc + i] = d[4 * nc + i] + eps;"),
    ("Psi path row index", "out[2 * nc + i] = d[4 * nc + i] - eps;", "out[2 * nc + i] = d[4 * i + 3] - eps;"),
    ("Psi y- taken at node k", "ym(Xm[(k + 1) * nxt + 6 * M->nb + j]);", "ym(Xm[k * nxt + 6 * M->nb + j]);"),
    ("parent joint torque sign", "Tq[p] = Tq[p] - cross2(rpx, rpy, lx, ly) - tau;",
     "Tq[p] = Tq[p] - cross2(rpx, rpy, lx, ly) + tau;"),
    ("parent joint force sign", "Fx[p] = Fx[p] - lx;", "Fx[p] = Fx[p] + lx;"),
    ("child anchor taken from parent",
     "const T& ly = u[nj + 2 * j + 1];\n    T rcx, rcy, rpx, rpy;\n    lever_arm(xt[3 * c + 2], M.jrho_c + 2 * j, rcx, rcy);",
     "const T& ly = u[nj + 2 * j + 1];\n    T rcx, rcy, rpx, rpy;\n    lever_arm(xt[3 * c + 2], M.jrho_p + 2 * j, rcx, rcy);"),
    ("Eq. (3) child anchor taken from parent",
     "lever_arm(xt[3 * c + 2], M.jrho_c + 2 * j, rcx, rcy);\n    lever_arm(xt[3 * p + 2], M.jrho_p + 2 * j, rpx, rpy);\n    // grad C_j",
     "lever_arm(xt[3 * c + 2], M.jrho_p + 2 * j, rcx, rcy);\n    lever_arm(xt[3 * p + 2], M.jrho_p + 2 * j, rpx, rpy);\n    // grad C_j"),
    ("cross product sign", "T cross2(const T& rx, const T& ry, const T& fx, const T& fy) { return rx * fy - ry * fx; }",
     "T cross2(const T& rx, const T& ry, const T& fx, const T& fy) { return ry * fx - rx * fy; }"),
    ("rotation transposed", "rx = c * rho[0] - s * rho[1];\n  ry = s * rho[0] + c * rho[1];",
     "rx = c * rho[0] + s * rho[1];\n  ry = -s * rho[0] + c * rho[1];"),
    ("gravity dropped", "Fy[b] = T(-M.mass[b] * M.g);", "Fy[b] = T(0.0);"),
    ("gravity sign", "Fy[b] = T(-M.mass[b] * M.g);", "Fy[b] = T(M.mass[b] * M.g);"),
    ("contact tangent sign", "const T ft = ltp - ltm;", "const T ft = ltm - ltp;"),
    ("inertia replaced by mass", "Tq[b] / M.inertia[b];", "Tq[b] / M.mass[b];"),
    ("q' = v index", "out[3 * b + k] = xt[3 * nb + 3 * b + k];", "out[3 * b + k] = xt[3 * nb + 3 * b];"),
    ("signed distance uses r_x", "contact_frame(M, xt[3 * b] + rx, xt[3 * b + 1] + ry);",
     "contact_frame(M, xt[3 * b] + rx, xt[3 * b + 1] + rx);"),
    ("friction cone sign", "sabs_plus(ltp + ltm - M.cmu[i] * ln)", "sabs_plus(ltp + ltm + M.cmu[i] * ln)"),
    ("penalty without ramp", "const T p = ramp(z);", "const T p = z;"),
    ("pseudo-Huber constant", "(p * p) / (1.0 + sqrt(1.0 + p * p))", "(p * p) / (2.0 + sqrt(1.0 + p * p))"),
    ("FOH weights swapped", "u[q] = (1.0 - tau) * uL[q] + tau * uR[q];",
     "u[q] = tau * uL[q] + (1.0 - tau) * uR[q];"),
    ("RK4 weights", "{1.0 / 6.0, 2.0 / 6.0, 2.0 / 6.0, 1.0 / 6.0}",
     "{1.0 / 8.0, 3.0 / 8.0, 3.0 / 8.0, 1.0 / 8.0}"),
    ("RK4 stage node", "{0.0, 0.5, 0.5, 1.0},", "{0.0, 0.5, 0.5, 0.5},"),
    ("RK4 stage coupling", "{{0.0}, {0.5}, {0.0, 0.5}, {0.0, 0.0, 1.0}}",
     "{{0.0}, {0.5}, {0.0, 0.5}, {0.0, 0.0, 0.5}}"),
    ("dilation dropped", "k[j][r] = s * fv[r];", "k[j][r] = fv[r];"),
    ("dual product rule term", "r.d[i] = a.v * b.d[i] + b.v * a.d[i];", "r.d[i] = a.v * b.d[i];"),
    ("dual sin derivative", "const double c = std::cos(a.v);", "const double c = -std::cos(a.v);"),
    ("dual sqrt derivative", "const double k = 0.5 / r.v;", "const double k = 1.0 / r.v;"),
    ("u_R seed column", "UR[q].d[nxt + nu + q] = 1.0;", "UR[q].d[nxt + q] = 1.0;"),
    ("s seed", "Sd.d[C - 1] = 1.0;", "Sd.d[C - 1] = 0.5;"),
    ("defect subtracts x_k", "defect[v + r] = x1[r] - X[(k + 1) * nxt + r];",
     "defect[v + r] = x1[r] - X[k * nxt + r];"),
    ("penalty subtracts y_{k+1}", "penalty[(size_t)k * nc + i] = x1[nx + i] - X[k * nxt + nx + i];",
     "penalty[(size_t)k * nc + i] = x1[nx + i] - X[(k + 1) * nxt + nx + i];"),
    ("VJP drops -rho on y_k", "gX[k * nxt + nx + i] -= rho[k * nc + i];", "gX[k * nxt + nx + i] -= 0.0;"),
    ("VJP node layout u_R", "double* gR = (layout == 0) ? gU + (k + 1) * nu",
     "double* gR = (layout == 0) ? gU + k * nu"),
    ("VJP node coupling", "gX[(k + 1) * nxt + r] -= w[k * nxt + r];", "gX[(k + 1) * nxt + r] += w[k * nxt + r];"),
    # node constraints (impact map and relaxed impulse conditions)
    ("joint impulse sign", "for (int r = 0; r < 2 * nj; ++r) lam[r] = -lam[r];",
     "for (int r = 0; r < 2 * nj; ++r) lam[r] = lam[r];"),
    ("grad C parent angle column", "G[(2 * j) * nq + 3 * p + 2] = G[(2 * j) * nq + 3 * p + 2] + rpy;",
     "G[(2 * j) * nq + 3 * p + 2] = G[(2 * j) * nq + 3 * p + 2] - rpy;"),
    ("K without M^-1", "acc = acc + G[r * nq + a] * minv[a] * G[c2 * nq + a];",
     "acc = acc + G[r * nq + a] * G[c2 * nq + a];"),
    ("impulse left out of w", "w[a] = vm[a] + minv[a] * Jphi[a];", "w[a] = vm[a];"),
    ("contact impulse moment", "Jphi[3 * b + 2] = Jphi[3 * b + 2] + cross2(crx[i], cry[i], ix, iy);",
     "Jphi[3 * b + 2] = Jphi[3 * b + 2] + cross2(crx[i], cry[i], iy, ix);"),
    ("pose continuity sign", "for (int a = 0; a < nq; ++a) g[a] = xp[a] - xm[a];",
     "for (int a = 0; a < nq; ++a) g[a] = xp[a] + xm[a];"),
    ("restitution dropped", "const T cn = vnp + e[i] * vnm;", "const T cn = vnp;"),
    ("tangential velocity from v-", "const T vtp = fr[i].tx * vxp + fr[i].ty * vyp;",
     "const T vtp = fr[i].tx * vxm + fr[i].ty * vym;"),
    ("normal velocity lever arm", "const T vyp = vp[3 * b + 1] + vp[3 * b + 2] * crx[i];",
     "const T vyp = vp[3 * b + 1] + vp[3 * b + 2] * cry[i];"),
    ("smooth-norm gradient", "(pt / sqrt(1.0 + pt * pt))", "(pt)"),
    ("Fischer-Burmeister sign", "return a + b - sqrt(a * a + b * b + delta);",
     "return a + b + sqrt(a * a + b * b + delta) - 2.0 * sqrt(delta);"),
    ("friction cone without mu", "const T rho = smooth_abs(M.cmu[i] * pn) - smooth_abs(pt);",
     "const T rho = smooth_abs(pn) - smooth_abs(pt);"),
    ("Gamma seed column", "gm[i].d[2 * nxt + 2 * nc + i] = 1.0;", "gm[i].d[2 * nxt + i] = 1.0;"),
    # full auxiliary state of Eq. (12)
    ("lambda_c without the rotation term", "const T vcx = xt[3 * nb + 3 * b] - xt[3 * nb + 3 * b + 2] * ry;",
     "const T vcx = xt[3 * nb + 3 * b];"),
    ("lambda_c lever arm", "const T vcx = xt[3 * nb + 3 * b] - xt[3 * nb + 3 * b + 2] * ry;",
     "const T vcx = xt[3 * nb + 3 * b] - xt[3 * nb + 3 * b + 2] * rx;"),
    ("phi_n state integrates phi_t", "out[6 * nb + 4 * i] = fn;", "out[6 * nb + 4 * i] = ft;"),
    ("rho_c without mu", "const T rho_c = smooth_abs(M.cmu[i] * fn) - smooth_abs(ft);",
     "const T rho_c = smooth_abs(fn) - smooth_abs(ft);"),
    ("cross penalty drops gamma", "sabs_plus(-fn) + sabs_plus(-phi) + sabs_plus(-gam) +",
     "sabs_plus(-fn) + sabs_plus(-phi) + sabs_plus(gam) +"),
    ("cross tangential force sign", "fx = fr.tx * ft + fr.nx * fn;", "fx = -(fr.tx * ft) + fr.nx * fn;"),
    # paper-faithful dynamics: Eq. (3) elimination, sinusoidal surface, RKF45
    ("Eq. (3) parent centripetal sign", "r[row] = wc * wc * rcx - wp * wp * rpx;",
     "r[row] = wc * wc * rcx + wp * wp * rpx;"),
    ("Eq. (3) centripetal term dropped", "r[row + 1] = wc * wc * rcy - wp * wp * rpy;",
     "r[row + 1] = T(0.0);"),
    ("Eq. (3) grad C child angle column", "{row, 3 * c + 2, -rcy}", "{row, 3 * c + 2, rcy}"),
    ("Eq. (3) grad C parent block", "{row + 1, 3 * p + 1, T(-1.0)}", "{row + 1, 3 * p + 1, T(1.0)}"),
    ("eliminated model parent torque sign", "      Tq[p] = Tq[p] - tau;\n      continue;",
     "      Tq[p] = Tq[p] + tau;\n      continue;"),
    ("eliminated model inertia", "K[(size_t)(3 * b + 2) * n + 3 * b + 2] = T(M.inertia[b]);",
     "K[(size_t)(3 * b + 2) * n + 3 * b + 2] = T(M.mass[b]);"),
    ("terrain normal sign", "f.nx = gx * inv;", "f.nx = -gx * inv;"),
    ("terrain slope uses sin", "const T gx = -(a * k) * cos(k * px);", "const T gx = -(a * k) * sin(k * px);"),
    ("signed distance not normalized", "f.phi = hc * inv;", "f.phi = hc;"),
    ("terrain tangent orientation", "f.ty = -f.nx;", "f.ty = f.nx;"),
    ("terrain force drops normal x", "fx = fr.tx * ft + fr.nx * ln;", "fx = fr.tx * ft;"),
    ("impact impulse in world axes", "const T ix = fr[i].tx * pt + fr[i].nx * pn;", "const T ix = pt;"),
    ("RKF45 coupling coefficient", "-845.0 / 4104.0}", "845.0 / 4104.0}"),
    ("RKF45 fourth-order weights",
     "{16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0,\n                         2.0 / 55.0}",
     "{25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0,\n                         0.0}"),
    ("RKF45 stage time", "{0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0}",
     "{0.0, 1.0 / 4.0, 3.0 / 8.0, 11.0 / 13.0, 1.0, 1.0 / 2.0}"),
    ("RKF45 selected as RK4", "return scheme == 1 ? kRKF45 : kRK4;", "return kRK4;"),
]


def _run_mutant(name, old, new):
    """Builds oracle.cpp with one planted error and runs the pin suites against
    it; returns (pytest return code, end of its output)."""
    src = open(SRC).read()
    if src.count(old) != 1:
        return None, f"mutation anchor not found once: {name}"
    with tempfile.TemporaryDirectory() as tmp:
        mpath = os.path.join(tmp, "oracle_mut.cpp")
        lpath = os.path.join(tmp, "liboracle_mut.so")
        open(mpath, "w").write(src.replace(old, new))
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", mpath,
                               "-o", lpath])
        env = dict(os.environ, CISCVX_ORACLE_LIB=lpath)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def mutant_results(request):
    """Runs every selected mutation once, several at a time (each is an
    independent compile plus a pytest subprocess), so the whole set takes
    about its total time divided by the host's cores."""
    selected = [it.callspec.params["name"] for it in request.session.items
                if getattr(it, "originalname", None) == "test_pins_reject_planted_error"]
    table = {m[0]: m for m in MUTATIONS}
    workers = max(1, min(len(selected), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {n: ex.submit(_run_mutant, *table[n]) for n in selected}
        return {n: f.result() for n, f in futs.items()}


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_reject_planted_error(name, old, new, mutant_results):
    rc, out = mutant_results[name] if name in mutant_results else _run_mutant(name, old, new)
    assert rc is not None, out
    assert rc != 0, f"pins did not catch: {name}\n{out}"


# Planted errors in the dense SOCP assembly (oracle/socp.py), caught by its pins.
SOCP_SRC = os.path.join(ROOT, "oracle", "socp.py")
SOCP_PINS = ["tests/test_oracle_socp.py"]
SOCP_MUTATIONS = [
    ("dynamics right-hand side takes the pre-impact state",
     "b_rows.append(jz - (lin[\"defect\"][k, r_] + Xp[k + 1, r_]))",
     "b_rows.append(jz - (lin[\"defect\"][k, r_] + Xm[k + 1, r_]))"),
    ("B+ placed on u_L", "r[uR] += lin[\"Bp\"][k, r_]", "r[uL] += lin[\"Bp\"][k, r_]"),
    ("impact slack sign", "r[L.col[\"nuGp\", k][r_]] -= 1.0", "r[L.col[\"nuGp\", k][r_]] += 1.0"),
    ("dynamics slack sign", "r[L.col[\"nuFm\", k][r_]] += 1.0", "r[L.col[\"nuFm\", k][r_]] -= 1.0"),
    ("Theta slack sign", "r[L.col[\"tth\", k][r_]] = -1.0\n            G_rows.append(r)\n            h_rows.append(hz)",
     "r[L.col[\"tth\", k][r_]] = 1.0\n            G_rows.append(r)\n            h_rows.append(hz)"),
    ("Psi sides swapped", "r[yp] += ps[\"J\"][k, r_, :ny]", "r[yp] += ps[\"J\"][k, r_, ny:]"),
    ("torque cost coupling", "P0[a, b_] += w / 3", "P0[a, b_] += w / 6"),
    ("proximal linear term sign", "c0[L.is_problem] = -prm[\"w_px\"] * zbar[L.is_problem]",
     "c0[L.is_problem] = prm[\"w_px\"] * zbar[L.is_problem]"),
    ("offset dropped from c", "c1 = D * (P0 @ o + c0)", "c1 = D * c0"),
    ("offset sign in b", "A1, b1 = A0 * D[None, :], b0 - A0 @ o", "A1, b1 = A0 * D[None, :], b0 + A0 @ o"),
    ("cone block scaled by the larger rho", "rG[r0:r0 + 2] = rG[r0:r0 + 2].min()",
     "rG[r0:r0 + 2] = rG[r0:r0 + 2].max()"),
    ("friction cone coefficient sign", "r[a] = -L.mu[i]", "r[a] = L.mu[i]"),
    ("second-order cone on the wrong input", "r1[pt] = -1.0", "r1[pn] = -1.0"),
    ("final boundary on the pre-impact state", "(L.col[\"xp\", N][:nx], prm[\"x_final\"])",
     "(L.col[\"xm\", N][:nx], prm[\"x_final\"])"),
]


def _run_socp_mutant(name, old, new, lib):
    """Runs the SOCP pins against a copy of the oracle package whose socp.py
    carries one planted error; returns (pytest return code, end of its output)."""
    src = open(SOCP_SRC).read()
    if src.count(old) != 1:
        return None, f"mutation anchor not found once: {name}"
    with tempfile.TemporaryDirectory() as tmp:
        # a tree whose oracle package carries the planted error; the built
        # oracle library and the product package are the real ones
        shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(tmp, "tests"),
                        ignore=shutil.ignore_patterns("__pycache__"))
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tmp, "oracle"),
                        ignore=shutil.ignore_patterns("__pycache__", "*.so", "*.lock"))
        os.symlink(os.path.join(ROOT, "paper_2604_09993_gb300"), os.path.join(tmp, "paper_2604_09993_gb300"))
        open(os.path.join(tmp, "oracle", "socp.py"), "w").write(src.replace(old, new))
        env = dict(os.environ, CISCVX_ORACLE_LIB=lib)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            *SOCP_PINS], cwd=tmp, env=env, capture_output=True, text=True, timeout=600)
        return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def socp_mutant_results(request, oracle_mod):
    """The selected SOCP mutations, several at a time (as mutant_results)."""
    selected = [it.callspec.params["name"] for it in request.session.items
                if getattr(it, "originalname", None) == "test_socp_pins_reject_planted_error"]
    table = {m[0]: m for m in SOCP_MUTATIONS}
    lib = oracle_mod.build()
    workers = max(1, min(len(selected), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {n: ex.submit(_run_socp_mutant, *table[n], lib) for n in selected}
        return {n: f.result() for n, f in futs.items()}


@pytest.mark.parametrize("name,old,new", SOCP_MUTATIONS, ids=[m[0] for m in SOCP_MUTATIONS])
def test_socp_pins_reject_planted_error(name, old, new, socp_mutant_results):
    rc, out = socp_mutant_results[name]
    assert rc is not None, out
    assert rc != 0, f"pins did not catch: {name}\n{out}"
    assert "passed" in out or "failed" in out, out
