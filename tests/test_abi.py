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


def test_struct_layouts_match_the_header(tmp_path):
    # the binding's ctypes mirrors of fim_stats and fim_db_desc against the C
    # compiler's view of include/fim.h: size and the offset of every field
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2412_19420_gb300 import fim
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fim.h"', 'int main(void) {']
    for st in (fim.fim_stats, fim.fim_db_desc):
        name = st.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        st, field, val = line.split()
        got[(st, field)] = int(val)
    for st in (fim.fim_stats, fim.fim_db_desc):
        name = st.__name__
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)


def test_binding_argument_counts_match_the_header():
    # every ctypes signature the binding declares has as many arguments as the
    # header's prototype of that entry point
    from paper_2412_19420_gb300 import fim
    txt = ""
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt += open(os.path.join(ROOT, "include", h)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(fim_\w+)\s*\(([^()]*)\)\s*;", txt):
        params = m.group(2).strip()
        protos[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    checked = 0
    for name, n in protos.items():
        f = getattr(fim._lib, name)
        if f.argtypes is None:
            continue
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)
        checked += 1
    assert checked >= 20


def test_flag_values_match_the_header():
    # every FIM_* flag the binding defines has the header's value
    from paper_2412_19420_gb300 import fim
    txt = open(os.path.join(ROOT, "include", "fim.h")).read()
    defs = {m.group(1): int(m.group(2), 16) for m in re.finditer(r"#define (FIM_\w+) (0x[0-9a-fA-F]+)u", txt)}
    for name in ("FIM_INPUT_DEVICE", "FIM_OUTPUT_DEVICE", "FIM_CSR_COMPACT", "FIM_STRICT", "FIM_LEARNED",
                 "FIM_PAIRS_POPC", "FIM_TRACE", "FIM_DIFFSET_RULE", "FIM_NO_SPLIT"):
        assert getattr(fim, name) == defs[name], name


def test_csr_format_from_element_sizes():
    # the binding marshals a CSR as wide (int64 offsets, int32 ids) or compact
    # (4-byte offsets, 2-byte ids) from the arrays' element sizes alone, and
    # rejects any other pairing rather than guessing
    import numpy as np
    from paper_2412_19420_gb300 import fim
    assert fim._csr_format(np.zeros(3, np.int64), np.zeros(2, np.int32)) == 0
    assert fim._csr_format(np.zeros(3, np.uint32), np.zeros(2, np.uint16)) == fim.FIM_CSR_COMPACT
    assert fim._csr_format(np.zeros(3, np.int32), np.zeros(0, np.int16)) == fim.FIM_CSR_COMPACT
    for ip, ix in ((np.int64, np.int16), (np.int32, np.int32), (np.uint8, np.uint8)):
        with pytest.raises(ValueError):
            fim._csr_format(np.zeros(3, ip), np.zeros(2, ix))
    try:
        import torch
    except ImportError:
        return
    assert fim._csr_format(torch.zeros(3, dtype=torch.int32), torch.zeros(2, dtype=torch.int16)) == \
        fim.FIM_CSR_COMPACT
    assert fim._csr_format(torch.zeros(3, dtype=torch.int64), torch.zeros(2, dtype=torch.int32)) == 0
