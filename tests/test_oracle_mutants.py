"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
at least one pin catches each.  The committed oracle source is never edited:
each mutant is a patched copy built into a temporary directory."""
import os
import subprocess

import pytest

import oracle as oracle_pkg
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle_pkg.__file__), "lloyd.c")

# (name, text in lloyd.c, replacement)
MUTANTS = [
    ("drop last coordinate", "for (int32_t j = 0; j < d; ++j) {\n    double t =",
     "for (int32_t j = 0; j < d - 1; ++j) {\n    double t ="),
    ("wrong sign in distance", "double t = (double)x[(int64_t)j * ld + i] - mu_k[j];",
     "double t = (double)x[(int64_t)j * ld + i] + mu_k[j];"),
    ("ties to highest index", "if (dc < bestd) { bestd = dc; best = c; }",
     "if (dc <= bestd) { bestd = dc; best = c; }"),
    ("transposed centroid index", "double dc = orc_sqdist(x, ld, i, d, mu + (int64_t)c * d);",
     "double dc = orc_sqdist(x, ld, i, d, mu + (int64_t)c);"),
    ("empty cluster zeroed", "mu_next[(int64_t)c * d + j] = mu_prev[(int64_t)c * d + j]; continue;",
     "mu_next[(int64_t)c * d + j] = 0.0; continue;"),
    ("mean divides by n+1", "sum / (double)cnt;", "sum / (double)(cnt + 1);"),
    ("last chunk dropped", "for (int64_t q = 0; q < nchunks; ++q) sum +=",
     "for (int64_t q = 0; q + 1 < nchunks; ++q) sum +="),
    ("sum over wrong coordinate", "s[(int64_t)zi * d + j] += (double)x[(int64_t)j * ld + i];",
     "s[(int64_t)zi * d + j] += (double)x[(int64_t)(d - 1 - j) * ld + i];"),
    ("E not squared", "double t = a[q] - b[q];\n    e2 = e2 + t * t;",
     "double t = a[q] - b[q];\n    e2 = e2 + fabs(t);"),
    ("non-strict stop", "if (esel < tol) { status = 0; break; }",
     "if (esel <= tol) { status = 0; break; }"),
    ("E_mode ignored", "double esel = e_mode == 1 ? e2 : sqrt(e2);", "double esel = sqrt(e2);"),
    ("labels from the new centroids", "    double* tmp = cur; cur = nxt; nxt = tmp;\n",
     "    double* tmp = cur; cur = nxt; nxt = tmp;\n    orc_assign(x, ld, n, d, k, cur, z, NULL);\n"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found uniquely: {name}"
    mut = tmp_path / "lloyd_mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "liblloyd_mut.so"
    subprocess.check_call(["gcc", *oracle_pkg.CFLAGS, str(mut), "-o", str(lib), "-lm"])
    orc = oracle_pkg.Oracle(str(lib))
    caught = []
    for pin in P.ALL_PINS:
        try:
            pin(orc)
        except (AssertionError, ValueError, IndexError, MemoryError) as e:
            caught.append((pin.__name__, type(e).__name__))
    assert caught, f"no pin caught the mutant '{name}'"
