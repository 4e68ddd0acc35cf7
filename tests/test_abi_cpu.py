"""The C-ABI library builds, loads without a GPU, and exports exactly what
include/mcpt.h declares (no compute calls: this runs on CPU-only hosts)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mcpt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcpt_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1409_2700_gb300 import _build
    return _build.build()


def test_header_matches_binding_exports():
    import paper_1409_2700_gb300 as M
    assert _declared() == sorted(M.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    syms = set(re.findall(r"\bT (mcpt_\w+)", out))
    for name in _declared():
        assert name in syms, name
    import paper_1409_2700_gb300 as M
    L = M.lib()
    for name in _declared():
        assert hasattr(L, name)


def test_library_is_sm103a_only(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    arches = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert arches == {"103a"}, arches


def test_create_without_gpu_fails_cleanly(libpath):
    """On a host with no usable GPU, mcpt_create reports ECUDA (no abort)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1409_2700_gb300 as M
    with pytest.raises(M.McptError) as ei:
        M.mcpt_create()
    assert ei.value.status == M.MCPT_ECUDA
    assert "device" in M.mcpt_last_error(None).lower()


def test_default_options(libpath):
    import paper_1409_2700_gb300 as M
    o = M.mcpt_default_options()
    assert o.precision == M.MCPT_FP64 and o.validate == 1 and o.wave_bytes == 1 << 30 and o.stream is None
    assert o.graphs == 1 and o.timing == 0 and o.mem_cap_bytes == 0
