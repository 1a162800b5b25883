"""Plant plausible mistakes in copies of the set-network oracle (on the CPU)
and check that at least one pin of tests/setnet_pins.py catches each.  The
committed oracle source is never edited: each mutant is a patched copy
imported from a temporary directory."""
import importlib.util
import os

import pytest

import setnet_pins as P
from oracle import setnet as sn_real

SRC = os.path.abspath(sn_real.__file__)

# (name, text in setnet.py, replacement)
MUTANTS = [
    ("no relu on h2", "h2 = np.maximum(z2, 0.0)", "h2 = z2"),
    ("no relu on h1", "h1 = np.maximum(z1, 0.0)", "h1 = z1"),
    ("no relu in the head", "a3 = np.maximum(z3, 0.0)", "a3 = z3"),
    ("max-pool instead of mean", "g = h2.mean(axis=1)", "g = h2.max(axis=1)"),
    ("sum-pool instead of mean", "g = h2.mean(axis=1)", "g = h2.sum(axis=1)"),
    ("sample std (ddof = 1)", "s = np.sqrt(((x - m[:, None, :]) ** 2).mean(axis=1))",
     "s = np.sqrt(((x - m[:, None, :]) ** 2).sum(axis=1) / (x.shape[1] - 1))"),
    ("constant coordinate std 0 kept", "s = np.where(s > 0, s, 1.0)", "s = np.where(s > 0, s, 1e-12)"),
    ("bias correction frozen at t = 1", "mh = m / (1 - beta1 ** t)\n        vh = v / (1 - beta2 ** t)",
     "mh = m / (1 - beta1)\n        vh = v / (1 - beta2)"),
    ("no bias correction", "mh = m / (1 - beta1 ** t)\n        vh = v / (1 - beta2 ** t)",
     "mh = m\n        vh = v"),
    ("second moment of g, not g^2", "v[...] = beta2 * v + (1 - beta2) * grads[n] ** 2",
     "v[...] = beta2 * v + (1 - beta2) * abs(grads[n])"),
    ("head bias dropped", "out = a3 @ W4.T + b4", "out = a3 @ W4.T"),
    ("transposed W2", "z2 = h1 @ W2.T + b2", "z2 = h1 @ W2 + b2"),
    ("backward mask of h2 dropped", 'dz2 = (dg[:, None, :] / S) * (cache["z2"] > 0)', "dz2 = dg[:, None, :] / S + 0 * cache['z2']"),
    ("backward mask of the head dropped", "dz3 = (dout @ W4) * (z3 > 0)", "dz3 = dout @ W4"),
    ("pool gradient not divided by S", 'dz2 = (dg[:, None, :] / S) * (cache["z2"] > 0)',
     'dz2 = dg[:, None, :] * (cache["z2"] > 0)'),
]


def _load_mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found uniquely: {old}"
    path = tmp_path / "setnet_mut.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"setnet_mut_{abs(hash(new))}", str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_real_oracle_passes_every_pin():
    for pin in P.ALL_PINS:
        pin(sn_real)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    mod = _load_mutant(tmp_path, old, new)
    caught = []
    for pin in P.ALL_PINS:
        try:
            pin(mod)
        except (AssertionError, ValueError, IndexError, FloatingPointError, ZeroDivisionError) as e:
            caught.append((pin.__name__, type(e).__name__))
    assert caught, f"no pin caught the mutant '{name}'"
