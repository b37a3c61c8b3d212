"""The tensor-core GEMM autotuner: it tunes every GEMM site of the sigma product, the tiles it
picks compute the same products as the default rule (parity with the oracle is unchanged),
and a tuning cache file written by one process is read back by the next (which then tunes
nothing).  Each case runs in a fresh process so that the process-wide table starts empty.
"""

import json
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = textwrap.dedent(
    """
    import json, sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import paper_2512_09811_gb300 as pp
    from oracle import pp_oracle as po
    from synth.inputs import make_inputs, random_vectors

    pp.load()
    inp = make_inputs(32, 128, 384, seed=3, mode="scaled")
    dot = pp.Dot(inp, order=2, prec=pp.PP_BF16)
    Z = random_vectors(4, 32, 128, seed=17)
    want = po.SigmaRef(inp.eps, inp.B, 32, order=2).sigma(Z)
    out = {{}}
    for name, prec in (("bf16", pp.PP_BF16), ("split", pp.PP_BF16X3)):
        got = dot.sigma(Z, prec=prec)
        out[name] = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    dot.close()
    out["report"] = pp.pp_autotune_report()
    print("RESULT " + json.dumps(out))
    """
)


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def _tunings(report):
    head = report.splitlines()[0]
    return int(head.split("tunings")[1])


def test_autotuner_tunes_every_site_and_keeps_parity(cuda_lib, tmp_path):
    cache = str(tmp_path / "tune.txt")
    off = _run({"PP_AUTOTUNE": "0"})
    on = _run({"PP_AUTOTUNE": "1", "PP_TUNE_CACHE": cache})
    again = _run({"PP_AUTOTUNE": "1", "PP_TUNE_CACHE": cache})
    assert _tunings(off["report"]) == 0 and "autotune off" in off["report"]
    assert _tunings(on["report"]) > 0
    for site in ("gamma", "U", "W", "KA", "EF", "KB", "slab", "sumP1", "sumP2"):
        assert any(ln.startswith(site + " ") for ln in on["report"].splitlines()), site
    # the cache written by the second process makes the third tune nothing, with the same table
    assert _tunings(again["report"]) == 0
    assert on["report"].splitlines()[1:] != [] and len(again["report"].splitlines()) == len(on["report"].splitlines())
    # same products whatever the tiles: the errors against the oracle agree to FP32 noise
    for name, bound in (("bf16", 1e-3), ("split", 1e-5)):
        assert on[name] <= bound and off[name] <= bound
        assert abs(on[name] - off[name]) <= 0.05 * off[name] + 1e-7
