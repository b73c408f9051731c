"""The C-ABI library loads and exports every symbol that include/agis.h declares (no GPU needed)."""
import ctypes as C
import os
import re

import paper_1112_4139_gb300 as pkg
from paper_1112_4139_gb300 import agis

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "agis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(agis_[a-z_0-9]+)\s*\(", src))


def test_library_builds_and_exports_all_declared_symbols():
    path = pkg.build()
    assert os.path.exists(path)
    lib = agis.load()
    declared = _declared()
    assert declared, "no declarations found"
    assert declared == set(agis.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert lib.agis_abi_version() == agis.ABI_VERSION == 8


def test_default_config_and_struct_sizes():
    assert C.sizeof(agis.BlockStats) == 104 and C.sizeof(agis.IterStats) == 3 * 104 + 80
    assert C.sizeof(agis.TuneEntry) == 32
    cfg = agis.default_config()
    assert cfg.precision == 0 and cfg.refresh_every == 8
    assert cfg.robust == 1 and cfg.n_rounds == 4 and cfg.n_eps == 3 and abs(cfg.lambda_att - 1e-3) < 1e-18
    assert cfg.seg_overlap == 12 and cfg.pivot_tol == 1e-12


def test_struct_layouts_of_the_full_calibration_model():
    # agis_config keeps its size (the calibration-model fields took its reserved words);
    # agis_obs gained the gate pointer
    assert C.sizeof(agis.Config) == 88
    assert C.sizeof(agis.Obs) == 8 * 8
    cfg = agis.default_config()
    assert cfg.cal_model == 0
