"""The oracle uses the constants the paper prints (tests/golden/paper_constants.txt)."""
import os

from oracle import kaiser_bessel, sara, sdmm
from paper_1307_4370_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_constants.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, value = line.split()[:2]
            vals[name] = float(value)
    return vals


def test_constants():
    c = load()
    assert sdmm.XI == c["xi"]
    assert sdmm.TAU == c["tau"]
    assert sdmm.BETA == c["beta"]
    assert kaiser_bessel.OVERSAMPLE == c["oversampling"]
    assert len(sara.ALL_BASES) == c["sara_bases"]
    assert all(w.isnr_db == c["isnr_db"] for w in inputs.WORKLOADS.values())
