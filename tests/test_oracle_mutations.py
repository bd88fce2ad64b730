"""The oracle's pins bite: each plausible mistake, planted in a scratch copy of the oracle (CPU only),
makes the pin tests fail. The real oracle is untouched."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("backward hop without complex conjugate", "a += conj(U[3 * j + i]) * v[j];", "a += U[3 * j + i] * v[j];"),
    ("backward hop without transpose", "a += conj(U[3 * j + i]) * v[j];", "a += conj(U[3 * i + j]) * v[j];"),
    ("forward link transposed", "a += U[3 * i + j] * v[j];", "a += U[3 * j + i] * v[j];"),
    ("staggered phase over one direction too many", "for (int nu = 0; nu < mu; ++nu) sum += c[nu];",
     "for (int nu = 0; nu <= mu; ++nu) sum += c[nu];"),
    ("long-link boundary sign on two slices only", "if (c[3] >= L[3] - 3) sl = -sl;", "if (c[3] >= L[3] - 2) sl = -sl;"),
    ("fat-link boundary sign dropped", "if (c[3] == L[3] - 1) sf = -sf;", "if (c[3] == L[3] - 99) sf = -sf;"),
    ("Naik backward hop of two sites", "shifted(L, c, mu, -3)", "shifted(L, c, mu, -2)"),
    ("backward link taken at the output site", "add_dag_mat_vec(out, link_at(fat, bwd1, mu), chi_at(ctx, bwd1), -1.0);",
     "add_dag_mat_vec(out, link_at(fat, idx, mu), chi_at(ctx, bwd1), -1.0);"),
    ("sign of D_eo D_oe in A", "y[i] = (4.0 * mass * mass + sigma) * x[i] - dd[i];",
     "y[i] = (4.0 * mass * mass + sigma) * x[i] + dd[i];"),
    ("mass term 2m instead of 4m^2", "y[i] = (4.0 * mass * mass + sigma) * x[i] - dd[i];",
     "y[i] = (2.0 * mass + sigma) * x[i] - dd[i];"),
    ("terms assigned instead of accumulated", "out[i] += s * a;", "out[i] = s * a;"),
    ("CG beta inverted", "double beta = rr_new / rr;", "double beta = rr / rr_new;"),
    ("multi-shift zeta without the shift difference", "(1.0 + dk * alpha)", "(1.0 + alpha)"),
]


@pytest.fixture(scope="module")
def scratch(tmp_path_factory):
    d = tmp_path_factory.mktemp("oracle_mutant")
    for sub in ("oracle", "hisq_inputs"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                        ignore=shutil.ignore_patterns("liboracle.so", "__pycache__", "*.tmp*"))
    os.makedirs(os.path.join(d, "tests"))
    for f in ("conftest.py", "test_oracle_dslash.py", "test_oracle_solvers.py", "test_oracle_smear.py",
              "test_oracle_ptc.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
    return str(d)


def run_pins(d, target="tests"):
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", target], cwd=d,
                         capture_output=True, text=True, timeout=600)
    return res.returncode, res.stdout[-400:]


def test_unmutated_copy_passes(scratch):
    rc, out = run_pins(scratch)
    assert rc == 0, out


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(scratch, name, old, new):
    src_path = os.path.join(scratch, "oracle", "oracle.c")
    original = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert old in original, "mutation anchor missing: " + old
    with open(src_path, "w") as f:
        f.write(original.replace(old, new, 1))
    lib = os.path.join(scratch, "oracle", "liboracle.so")
    if os.path.exists(lib):
        os.remove(lib)
    try:
        rc, out = run_pins(scratch)
        assert rc != 0, "pins did not catch: " + name
    finally:
        with open(src_path, "w") as f:
            f.write(original)
        if os.path.exists(lib):
            os.remove(lib)


SMEAR_MUTATIONS = [
    ("backward step without the dagger", "M = M @ np.conj(np.swapaxes(U[at, d], -1, -2))", "M = M @ U[at, d]"),
    ("backward step takes the link at the starting site",
     "at = _shift_index(L, d, -1, at)\n            M = M @ np.conj(np.swapaxes(U[at, d], -1, -2))",
     "M = M @ np.conj(np.swapaxes(U[at, d], -1, -2))\n            at = _shift_index(L, d, -1, at)"),
    ("five-link staple closed in crossed order", "(mu, 1), (nu, -s), (rho, -r)]", "(mu, 1), (rho, -r), (nu, -s)]"),
    ("seven-link staple returning on the wrong side", "(rho, -r), (sigma, -q)]", "(rho, -r), (sigma, q)]"),
    ("Lepage term displaced one site only", "paths[\"lepage\"].append([(nu, s), (nu, s), (mu, 1), (nu, -s), (nu, -s)])",
     "paths[\"lepage\"].append([(nu, s), (mu, 1), (nu, -s)])"),
    ("Naik link of two hops", "[(mu, 1), (mu, 1), (mu, 1)]", "[(mu, 1), (mu, 1)]"),
    ("projection by (W^dag W)^(1/2)", "(1.0 / np.sqrt(lam))", "np.sqrt(lam)"),
    ("projection factor on the wrong side", "return W @ inv_sqrt", "return inv_sqrt @ W"),
]


@pytest.mark.parametrize("name,old,new", SMEAR_MUTATIONS, ids=[m[0] for m in SMEAR_MUTATIONS])
def test_smear_mutation_is_caught(scratch, name, old, new):
    src_path = os.path.join(scratch, "oracle", "smear.py")
    original = open(os.path.join(ROOT, "oracle", "smear.py")).read()
    assert old in original, "mutation anchor missing: " + old
    with open(src_path, "w") as f:
        f.write(original.replace(old, new, 1))
    try:
        rc, out = run_pins(scratch, "tests/test_oracle_smear.py")
        assert rc != 0, "pins did not catch: " + name
    finally:
        with open(src_path, "w") as f:
            f.write(original)


PTC_MUTATIONS = [
    ("backward transport without the conjugate", 'return np.einsum("nji,nj->ni", fat[n, mu].conj(), psi[n])',
     'return np.einsum("nji,nj->ni", fat[n, mu], psi[n])'),
    ("forward transport from the backward neighbour", "n = neighbours(L, mu, +1)", "n = neighbours(L, mu, -1)"),
    ("adjoint transport taken as the transport itself", "return transport(L, fat, psi, h + 4 if h <= 4 else h - 4)",
     "return transport(L, fat, psi, h)"),
    ("weight gradient without the conjugate input", 'gW = np.einsum("bhvc,avc->abh", u.conj(), g_out)',
     'gW = np.einsum("bhvc,avc->abh", u, g_out)'),
    ("input gradient without the conjugate weights", 'mixed = np.einsum("abh,avc->bhvc", W.conj(), g_out)',
     'mixed = np.einsum("abh,avc->bhvc", W, g_out)'),
    ("loss gradient not averaged over pairs", "g2 = to_full(L, even=e / nx / n)[None]", "g2 = to_full(L, even=e / nx)[None]"),
    ("tied layer 2 without the conjugate", "W2[0, a, h] = np.conj(W1[a, 0, adjoint_hop(h)])",
     "W2[0, a, h] = W1[a, 0, adjoint_hop(h)]"),
]


@pytest.mark.parametrize("name,old,new", PTC_MUTATIONS, ids=[m[0] for m in PTC_MUTATIONS])
def test_ptc_mutation_is_caught(scratch, name, old, new):
    src_path = os.path.join(scratch, "oracle", "ptc.py")
    original = open(os.path.join(ROOT, "oracle", "ptc.py")).read()
    assert old in original, "mutation anchor missing: " + old
    with open(src_path, "w") as f:
        f.write(original.replace(old, new, 1))
    try:
        rc, out = run_pins(scratch, "tests/test_oracle_ptc.py")
        assert rc != 0, "pins did not catch: " + name
    finally:
        with open(src_path, "w") as f:
            f.write(original)
