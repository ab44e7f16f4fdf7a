"""The C ABI library loads and exports every entry point include/fim.h declares
(no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fim_\w+)\s*\(", txt))
    return names - {"fim_ctx"}


@pytest.fixture(scope="module")
def lib():
    from paper_2412_19420_gb300 import build
    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 16
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_host_only_calls():
    from paper_2412_19420_gb300 import fim
    assert fim.fim_version() >> 16 == 1
    assert fim.fim_minsup_from_ppm(10_000, 10_000) == 100
    assert fim.fim_minsup_from_ppm(12_345, 20_000) == 247
    assert fim.fim_minsup_from_ppm(0, 5) == 1
    assert fim.fim_minsup_from_ppm(10, 0) == 1
    assert "wait" in fim.fim_strerror(fim.FIM_E_TIMEOUT)
    assert "invariant" in fim.fim_strerror(fim.FIM_E_CHECK)
    assert fim.fim_strerror(12345) == "unknown status"


def test_no_device_is_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2412_19420_gb300 import fim
    with pytest.raises(fim.FimError) as e:
        fim.fim_create(0)
    assert e.value.code == fim.FIM_E_NODEV
