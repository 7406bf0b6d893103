"""The C-ABI library loads and exports every entry point include/sf.h declares
(no compute call: this runs without a GPU)."""
import os
import re

import pytest

from paper_2605_08528_b300 import build as B
from paper_2605_08528_b300 import sf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sf_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    B.build()
    L = sf.lib()
    names = declared("sf.h")
    assert "sf_step" in names and "sf_reset" in names and "sf_load_roads" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert sf.sf_version().startswith("sf ")


def test_binding_names_match_the_abi():
    for n in declared("sf.h"):
        if n.endswith("last_error"):   # message accessors, used inside the binding
            continue
        assert hasattr(sf, n), n


def test_create_without_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sf.SFError) as e:
        sf.sf_create()
    assert e.value.status == sf.SF_ERR_CUDA


def test_obs_layout_constants():
    assert sf.OBS_DIM == 16 + 8 * 10 + 32 * 7


def test_world_range_is_validated_before_any_device_call():
    for bad in [(3, 2), (-1, 4), (2, 0), (2, 2)]:
        with pytest.raises(sf.SFError) as e:
            sf.sf_create(world_range=bad)
        assert e.value.status == sf.SF_ERR_INVALID_ARG, bad


def test_weather_model_is_validated_before_any_device_call():
    with pytest.raises(sf.SFError) as e:
        sf.sf_create(weather_model=2)
    assert e.value.status == sf.SF_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["sf_config", "sf_roads", "sf_outputs", "sf_metrics", "sf_lf_outputs",
                                  "sf_ppo_config", "sf_ppo_rollout"])
def test_struct_layout_matches_the_header(tmp_path, name):
    """Each ctypes mirror of a C struct of include/sf.h has the C struct's size and
    field offsets (a small C program compiled here prints them)."""
    import ctypes
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    S = getattr(sf, name)
    fields = [n for n, *_ in S._fields_]
    prog = tmp_path / "m.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sf.h"\nint main(void) {\n'
                    '  printf("%%zu", sizeof(%s));\n' % name +
                    "".join('  printf(" %%zu", offsetof(%s, %s));\n' % (name, n) for n in fields) +
                    "  return 0;\n}\n")
    exe = tmp_path / "m"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(S)
    assert out[1:] == [getattr(S, n).offset for n in fields]


def test_metrics_calls_reject_a_null_handle():
    L = sf.lib()
    assert L.sf_get_metrics(None, None) == sf.SF_ERR_INVALID_ARG
    assert L.sf_reset_metrics(None) == sf.SF_ERR_INVALID_ARG
