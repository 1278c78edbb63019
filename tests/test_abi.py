"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no compute call: this runs without a GPU)."""
from __future__ import annotations

import glob
import os
import re

from paper_1903_06838_gb300 import pd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pd_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_entry_points()
    assert {"pd_create", "pd_process", "pd_process_host", "pd_destroy",
            "pd_get_summary", "pd_reset_summary", "pd_strerror"} <= names


def test_library_loads_and_exports_every_declared_symbol():
    pd.build()
    lib = pd.load()
    exported = pd.exported_symbols()
    missing = declared_entry_points() - exported
    assert not missing, missing
    for name in declared_entry_points():
        assert hasattr(lib, name)


def test_error_strings_without_gpu():
    pd.load()
    assert pd.pd_strerror(pd.PD_OK) == "ok"
    assert pd.pd_strerror(pd.PD_EALIGN).startswith("misaligned")
    assert pd.pd_strerror(pd.PD_EOVERFLOW) == "hit capacity exceeded"


def test_create_validates_before_touching_the_device():
    """pd_create's argument checks run before any CUDA call, so they can be
    exercised here: invalid input gives PD_EINVAL, valid input (including
    every golden-case geometry) passes validation and only then meets the
    device (which, without a GPU, fails with a CUDA or memory error)."""
    import numpy as np
    import pytest
    from tests._cases import load_cases
    for case in load_cases():
        try:
            ctx = pd.pd_create(case["geometry"], case["ped_arr"], case["gain_arr"],
                               case["thresholds"])
        except pd.PdError as e:
            assert e.code in (pd.PD_ECUDA, pd.PD_ENOMEM), e
        else:  # a GPU is present
            pd.pd_destroy(ctx)
    g = dict(n_modules=1, rows=4, cols=6, unit_rows=4, unit_cols=4, cm_mode=0)
    t = dict(cm_cut_adu=1.0, zero_thr_kev=0.5, seed_thr_kev=0.5, photon_kev=1.0)
    z = np.zeros(24, np.float32)
    with pytest.raises(pd.PdError) as ei:
        pd.pd_create(g, z, z, t)
    assert ei.value.code == pd.PD_EINVAL
    for bad in (dict(t, zero_thr_kev=2.0), dict(t, photon_kev=0.0),
                dict(t, zero_thr_kev=-1.0), dict(t, hist_bins=5000)):
        with pytest.raises(pd.PdError) as ei:
            pd.pd_create(dict(g, cols=8), np.zeros(32, np.float32),
                         np.zeros(32, np.float32), bad)
        assert ei.value.code == pd.PD_EINVAL
