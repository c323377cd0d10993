"""The oracle's pins catch plausible mistakes.

Each case copies the oracle's C source, plants one mistake of the kind a
restatement of the paper could contain (a dropped term, a wrong sign, a
wrong index or bit order, a transposed operand, an off-by-one, a wrong tie
rule), compiles the copy on the CPU and runs the pin suite against it: the
suite must fail.  The oracle itself is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cashash_oracle.c")

MUTANTS = {
    "centring sign": ("double t = (double)x[j] - mu[j];", "double t = (double)x[j] + mu[j];"),
    "dropped projection term": ("for (int j = 0; j < ORACLE_DIM; ++j) {\n    double t",
                                "for (int j = 0; j < ORACLE_DIM - 1; ++j) {\n    double t"),
    "sign at zero": ("if (v > 0.0) c[b >> 5]", "if (v >= 0.0) c[b >> 5]"),
    "bucket bit order": ("if (v > 0.0) id |= 1u << i;", "if (v > 0.0) id |= 1u << (m - 1 - i);"),
    "table rows transposed": ("R + (uint64_t)(nb + t * m + i) * ORACLE_DIM",
                              "R + (uint64_t)(nb + i * T + t) * ORACLE_DIM"),
    "code word layout": ("c[b >> 5] |= 1u << (b & 31);", "c[b & 3] |= 1u << (b >> 2);"),
    "mean divisor": ("(double)s[j] / (double)n;", "(double)s[j] / (double)(n + 1);"),
    "dropped code word": (" + __builtin_popcount(a[3] ^ b[3])", ""),
    "rank tie order": ("if (a->j != b->j) return a->j < b->j ? -1 : 1;\n  return 0;\n}\n\ntypedef struct {\n  int32_t d;",
                       "if (a->j != b->j) return a->j > b->j ? -1 : 1;\n  return 0;\n}\n\ntypedef struct {\n  int32_t d;"),
    "ratio not strict": ("if (lhs < rhs) mj", "if (lhs <= rhs) mj"),
    "L1 distance": ("s += e * e;", "s += e < 0 ? -e : e;"),
    "no dedup": ("if (seen[j] == q) continue;", ""),
    "k off by one": ("nc < K ? nc : K;", "nc < K ? nc : K - 1;"),
    "F transposed": ("const double a = (F[0] * x + F[1] * y) + F[2];\n  const double b = (F[3] * x + F[4] * y) + F[5];\n  const double c = (F[6] * x + F[7] * y) + F[8];",
                     "const double a = (F[0] * x + F[3] * y) + F[6];\n  const double b = (F[1] * x + F[4] * y) + F[7];\n  const double c = (F[2] * x + F[5] * y) + F[8];"),
    "distance order": ("if (a->d != b->d) return a->d < b->d ? -1 : 1;", "if (a->d != b->d) return a->d > b->d ? -1 : 1;"),
    "tau inclusive": ("if (cand[e].h <= p->tau)", "if (cand[e].h < p->tau)"),
    "mutual reverse F not transposed": ("Ft[3 * u + v] = J->F[9 * (size_t)i + 3 * v + u];",
                                        "Ft[3 * u + v] = J->F[9 * (size_t)i + 3 * u + v];"),
    "mutual check dropped": ("if (m[q] >= 0 && mr[m[q]] != (int32_t)q) m[q] = -1;", ""),
    "single accepted without the flag": ("} else if (ntop == 1 && (p->flags & ORACLE_ACCEPT_SINGLE)) {",
                                         "} else if (ntop == 1) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found exactly once: %s" % name
    mut = src.replace(old, new)
    c = tmp_path / "mutant.c"
    c.write_text(mut)
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                    "-I", os.path.join(ROOT, "oracle"), "-o", str(so), str(c)], check=True)
    env = dict(os.environ, CASHASH_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and " failed" in r.stdout, "pins did not catch mutant '%s'" % name


GA_SRC = os.path.join(ROOT, "oracle", "ga.py")

GA_MUTANTS = {
    "design rows transposed": ('np.einsum("ni,nj->nij", xb, xa)', 'np.einsum("ni,nj->nij", xa, xb)'),
    "rank 2 not enforced": ("S[2] = 0.0", "S[2] = S[2]"),
    "normalisation scale": ("s = np.sqrt(2.0) / md", "s = 1.0 / md"),
    "Sampson term dropped": (" + Ftx[:, 1] ** 2", ""),
    "ties to the later hypothesis": ("if cnt > best:", "if cnt >= best:"),
    "samples may repeat": ("if p <= v:", "if p < v:"),
    "acceptance not inclusive": ("gp.inlier_den * n_in >= gp.inlier_num * m", "gp.inlier_den * n_in > gp.inlier_num * m"),
    "no refit": ("if np.count_nonzero(inl) >= 8:", "if False:"),
    "selection ties to the higher index": ("np.lexsort((np.arange(n), -s.astype(np.float64)))",
                                           "np.lexsort((-np.arange(n), -s.astype(np.float64)))"),
    "subset size rounded down": ("k = (n * pct + 99) // 100", "k = (n * pct) // 100"),
    "stop rule with w^6": ("base = 1.0 - w4 * w4", "base = 1.0 - w4 * w2"),
    "stop rule on the hypotheses before the batch": ("ransac_stop(best, m, done, gp.confidence)",
                                                     "ransac_stop(best, m, done - BATCH, gp.confidence)"),
}


@pytest.mark.parametrize("name", sorted(GA_MUTANTS))
def test_ga_pins_reject_mutant(name, tmp_path):
    old, new = GA_MUTANTS[name]
    src = open(GA_SRC).read()
    assert src.count(old) == 1, "mutation anchor not found exactly once: %s" % name
    mut = tmp_path / "ga_mutant.py"
    mut.write_text(src.replace(old, new))
    env = dict(os.environ, CASHASH_ORACLE_GA=str(mut))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_ga.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and " failed" in r.stdout, "pins did not catch mutant '%s'" % name
