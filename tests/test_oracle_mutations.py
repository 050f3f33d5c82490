"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of the
oracle's C source (a flipped sign, a wrong index, a dropped factor, a transposed operand, a
swapped basis function) or of its Python part (the Dirichlet split, the null space, the error
norm, a rule weight), and runs the fast pins against it in a child process, which must fail;
the unchanged oracle must pass.

Pins run: the DG closed form and the embedding identity, the invariants (symmetry, A 1 = 0,
rigid motions), the load vector's closed form, the singular rule's closed form and polar
evaluation, the clip tests (both balls), the label-dependent and tabulated kernels' closed
forms, the row-wise reproduction of -Delta and the Sec. 3.1 rates.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

from oracle import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PINS = [
    "tests/test_oracle_dg.py::test_dg_singular_rule_constant_kernel_closed_form",
    "tests/test_oracle_dg.py::test_continuous_matrix_is_the_restriction_of_the_dg_matrix",
    "tests/test_oracle_system.py::test_invariants",
    "tests/test_oracle_system.py::test_bfs_pairs_equal_brute_force",
    "tests/test_oracle_system.py::test_load_vector_closed_form_for_linear_f",
    "tests/test_oracle_duffy.py",
    "tests/test_oracle_clip.py",
    "tests/test_oracle_clip_square.py",
    "tests/test_oracle_materials.py",
    "tests/test_oracle_tabulated.py",
    "tests/test_oracle_system.py::test_constant_kernel_reproduces_laplacian_rowwise",
    "tests/test_oracle_system.py::test_paper_E1_fractional_rates",
    "tests/test_oracle_system.py::test_peridynamic_kernel_reproduces_navier_rowwise",
    "tests/test_oracle_system.py::test_l2_error_closed_forms",
    "tests/test_oracle_neumann.py",
    "tests/test_oracle_rules.py",
]

# (name, text of the oracle source, the same text with the mistake)
MUTATIONS = [
    ("inner basis sign", "for (int b = 0; b < 3; ++b) D[posl[b]] -= Q[b];",
     "for (int b = 0; b < 3; ++b) D[posl[b]] += Q[b];"),
    ("inner basis index", "for (int b = 0; b < 3; ++b) D[posl[b]] -= Q[b];",
     "for (int b = 0; b < 3; ++b) D[b] -= Q[b];"),
    ("sub-triangle Jacobian dropped", "double w = ap * (P->ri.w[q] * dT);",
     "double w = ap * P->ri.w[q];"),
    ("basis of the wrong element", "else barycentric(Vl, yx, yy, Q);",
     "else barycentric(Vk, yx, yy, Q);"),
    ("kernel exponent sign", "return P->c * pow(r2, -1.0 - P->s);",
     "return P->c * pow(r2, -1.0 + P->s);"),
    ("peridynamic tensor component", "G[1] = P->c * zx * zy / r3;",
     "G[1] = P->c * zx * zx / r3;"),
    ("cap centre on the wrong side",
     "out[m][0] = cx + delta * (qy / len);\n                    out[m][1] = cy + delta * (-qx / len);",
     "out[m][0] = cx + delta * (-qy / len);\n                    out[m][1] = cy + delta * (qx / len);"),
    ("edge-pair Duffy weight", "wq * scale * xi * xi * L * wr", "wq * scale * xi * L * wr"),
    ("vertex-pair Duffy basis", "D[upos[3]] = -y1 * (1.0 - w2);", "D[upos[3]] = -y1 * w2;"),
    ("identical-pair Duffy difference", "D1 = xi * (h2 - h1)", "D1 = xi * (h1 - h2)"),
    ("DG split basis transposed",
     "D[lpos[0]] = -(1.0 - y1); D[lpos[1]] = -(y1 - y2); D[lpos[2]] = -y2;",
     "D[lpos[0]] = -(1.0 - y1); D[lpos[1]] = -y2; D[lpos[2]] = -(y1 - y2);"),
    ("load vector basis transposed", "+= ap * fx * P.ro.l[p][a];", "+= ap * fx * P.ro.l[p][(a + 1) % 3];"),
    ("outer point map", "*x = (l[0] * V[0][0] + l[1] * V[1][0]) + l[2] * V[2][0];",
     "*x = (l[0] * V[0][0] + l[2] * V[1][0]) + l[1] * V[2][0];"),
    ("material of the wrong element", "fm = mscale[mat[S->pairs[2 * pq]] * nmat + mat[S->pairs[2 * pq + 1]]];",
     "fm = mscale[mat[S->pairs[2 * pq]] * nmat + mat[S->pairs[2 * pq]]];"),
    ("table interpolation weight", "double w = t - i;", "double w = 1.0 - (t - i);"),
    ("square clip half-plane", "n = sh_pass(B, n, 1, -1.0, delta, A);", "n = sh_pass(B, n, 1, 1.0, delta, A);"),
    ("circle crossing root", "t2 = (-B + r) / A;", "t2 = (B + r) / A;"),
    ("edge quadratic term", "double B = ex * ux + ey * uy;", "double B = ex * ux - ey * uy;"),
    ("vertex on the circle", "inside[a] = (dx * dx + dy * dy) <= delta2;", "inside[a] = (dx * dx + dy * dy) < delta2;"),
    ("peridynamic kernel power", "double r3 = r2 * sqrt(r2);", "double r3 = r2 * r2;"),
    ("traversal stops after the first layer", "{ ivec_push(&queue, l); ivec_push(res, l); }",
     "{ if (e == k) ivec_push(&queue, l); ivec_push(res, l); }"),
]


# mistakes in the oracle's Python part: (file of the oracle package, name, text, mistake)
PY_MUTATIONS = [
    ("oracle.py", "Dirichlet column split sign", "b = system.F[free] - A[free][:, dof_d] @ g[dof_d]",
     "b = system.F[free] + A[free][:, dof_d] @ g[dof_d]"),
    ("oracle.py", "rotation mode of the null space", "Z[:, 0, 2] = -X[:, 1]", "Z[:, 0, 2] = X[:, 1]"),
    ("oracle.py", "L2 error Jacobian", "err += np.sum(w * det *", "err += np.sum(w * 0.5 * det *"),
    ("rules.py", "7-point rule weight", "(third, third, third, 27.0 / 120.0)", "(third, third, third, 27.0 / 60.0)"),
]


def _run_pins(job):
    """The pins in a child process against a copy of the oracle package (the child's working
    directory holds it, so it is imported first) and a build of the oracle's C source."""
    cwd, lib = job
    env = dict(os.environ, NLFEM_ORACLE_LIB=lib, OMP_NUM_THREADS="2", PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-W", "ignore", "-m", "not gpu"]
    return subprocess.run(cmd + [os.path.join(ROOT, p) for p in PINS], cwd=cwd, env=env,
                          capture_output=True, text=True, timeout=900)


def _package_copy(root, mutation=None):
    pkg = os.path.dirname(orc.SRC)
    d = root / "oracle"
    d.mkdir(parents=True)
    for f in ("__init__.py", "oracle.py", "rules.py"):
        t = open(os.path.join(pkg, f)).read()
        if mutation and f == mutation[0]:
            assert t.count(mutation[2]) == 1, f"mutation site not unique or missing: {mutation[2]!r}"
            t = t.replace(mutation[2], mutation[3])
        (d / f).write_text(t)
    return str(root)


def test_planted_mistakes_fail_a_pin_and_the_oracle_passes(tmp_path):
    text = open(orc.SRC).read()
    base = _package_copy(tmp_path / "base")
    jobs = []                                    # (name, C source text, package directory)
    jobs.append(("unchanged", text, base))
    for name, old, new in MUTATIONS:
        assert text.count(old) == 1, f"mutation site not unique or missing: {old!r}"
        jobs.append((name, text.replace(old, new), base))
    for i, mu in enumerate(PY_MUTATIONS):
        jobs.append((mu[1], text, _package_copy(tmp_path / f"py{i}", mu)))
    built = {}
    runs_in = []
    for i, (name, src_text, cwd) in enumerate(jobs):
        if src_text not in built:
            src = tmp_path / f"v{i}.c"
            src.write_text(src_text)
            built[src_text] = str(tmp_path / f"libv{i}.so")
            orc.compile_source(str(src), built[src_text])
        runs_in.append((cwd, built[src_text]))
    # the children run in parallel (each pin run stops at its first failure)
    with ThreadPoolExecutor(max_workers=max(1, min(6, (os.cpu_count() or 2) // 2))) as ex:
        runs = list(ex.map(_run_pins, runs_in))
    assert runs[0].returncode == 0, runs[0].stdout[-2000:]
    missed = [name for (name, _, _), r in zip(jobs[1:], runs[1:]) if r.returncode != 1]
    assert not missed, f"no pin failed for: {missed}"
