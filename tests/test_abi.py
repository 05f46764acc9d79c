"""The C-ABI library: builds, loads and exports what include/lp.h declares.

No GPU: only calls that fail in host-side validation are made here.
"""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lp():
    from paper_2401_11415_gb300 import _build
    _build.build()
    import paper_2401_11415_gb300 as m
    return m


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lp_\w+)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol(lp):
    names = declared_functions()
    assert "lp_graph_create" in names and "lp_predict" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lp.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lp_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = lp.lib()
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_options(lp):
    assert "sm_103a" in lp.lp_version()
    assert lp.lp_get_option(lp.LP_OPT_WARP_MAX_WEDGES) == 256
    assert lp.lp_get_option(lp.LP_OPT_MED_MAX_WEDGES) == 1024
    old = lp.lp_get_option(lp.LP_OPT_SPLIT_TARGET)
    lp.lp_set_option(lp.LP_OPT_SPLIT_TARGET, 4096)
    assert lp.lp_get_option(lp.LP_OPT_SPLIT_TARGET) == 4096
    lp.lp_set_option(lp.LP_OPT_SPLIT_TARGET, old)
    with pytest.raises(lp.LPError) as e:
        lp.lp_set_option(lp.LP_OPT_WARP_MAX_WEDGES, 100000)
    assert e.value.status == lp.LP_EINVAL
    assert lp.lp_get_option(lp.LP_OPT_BIG_CTA_THREADS) == 1024
    with pytest.raises(lp.LPError) as e:
        lp.lp_set_option(lp.LP_OPT_BIG_CTA_THREADS, 768)
    assert e.value.status == lp.LP_EINVAL
    assert lp.lp_get_option(99) == -1


def test_host_validation_rejects_bad_csr(lp):
    import numpy as np
    bad = [
        (3, [0, 1, 2, 1], [1, 0]),           # decreasing offsets
        (2, [1, 1, 2], [0, 1]),              # offsets[0] != 0
        (2, [0, 1, 2], [1, 5]),              # index out of range
        (2, [0, 1, 2], [0, 0]),              # self-loop
        (3, [0, 2, 3, 4], [1, 1, 0, 0]),     # duplicate arc
    ]
    for n, off, idx in bad:
        with pytest.raises(lp.LPError) as e:
            lp.lp_graph_create(n, np.array(off, np.int32), np.array(idx, np.int32))
        assert e.value.status == lp.LP_EINVAL, (off, idx)
        assert lp.lp_last_error()


def test_stats_struct_matches_header(lp):
    text = open(os.path.join(ROOT, "include", "lp.h")).read()
    body = text[text.index("typedef struct {\n  int64_t wedges"):text.index("} lp_stats;")]
    fields = re.findall(r"\b(?:int64_t|int32_t|float)\s+([\w, \[\]0-9]+);", body)
    names = [re.sub(r"\[\d+\]", "", x).strip() for f in fields for x in f.split(",")]
    assert names == [f for f, _ in lp.lp_stats._fields_]


def test_no_cpu_fallback_in_binding():
    src = open(os.path.join(ROOT, "paper_2401_11415_gb300", "__init__.py")).read()
    assert "import oracle" not in src and "lp_inputs" not in src
