"""The C-ABI library builds, loads and exports every entry point of
include/ngb.h; the Python structures match the C layout (CPU only, no GPU
calls)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2007_14236_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ngb.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"NGB_API\s+[\w\s\*]+?\b(ngb_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    try:
        return B.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ngb_create", "ngb_add_population", "ngb_connect", "ngb_simulate", "ngb_get_spikes",
                     "ngb_destroy", "ngb_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(ngb_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        assert getattr(lib, n) is not None
    # nothing but the ABI leaks out
    assert all(n.startswith("ngb_") for n in exported)


def test_binding_lists_every_symbol():
    from paper_2007_14236_gb300 import ngb
    assert sorted(ngb.EXPORTS) == _declared()


def test_struct_layouts_match_c(tmp_path):
    from paper_2007_14236_gb300 import ngb
    src = tmp_path / "layout.c"
    structs = {"ngb_sim_config": ngb.SimConfig, "ngb_poisson_drive": ngb.PoissonDrive,
               "ngb_lif_params": ngb.LifParams, "ngb_aeif_params": ngb.AeifParams, "ngb_conn_spec": ngb.ConnSpec,
               "ngb_dist_spec": ngb.DistSpec, "ngb_syn_spec": ngb.SynSpec, "ngb_stats": ngb.Stats,
               "ngb_stdp_params": ngb.StdpParams}
    body = "".join('printf("%s %%zu\\n", sizeof(%s));\n' % (k, k) for k in structs)
    body += 'printf("aeif_poisson %zu\\n", offsetof(ngb_aeif_params, poisson));\n'
    body += 'printf("cfg_stream %zu\\n", offsetof(ngb_sim_config, stream));\n'
    body += 'printf("aeif_ports %zu\\n", offsetof(ngb_aeif_params, n_ports));\n'
    body += 'printf("aeif_tau_decay %zu\\n", offsetof(ngb_aeif_params, tau_decay_ms));\n'
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ngb.h"\nint main(void){\n%s return 0;}\n' % body)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.split("\n") if line)
    for k, cls in structs.items():
        assert int(got[k]) == ctypes.sizeof(cls), k
    assert int(got["aeif_poisson"]) == ngb.AeifParams.poisson.offset
    assert int(got["cfg_stream"]) == ngb.SimConfig.stream.offset
    assert int(got["aeif_ports"]) == ngb.AeifParams.n_ports.offset
    assert int(got["aeif_tau_decay"]) == ngb.AeifParams.tau_decay_ms.offset


def test_invalid_arguments_fail_without_touching_a_gpu(libpath):
    from paper_2007_14236_gb300 import ngb
    L = ngb.load(build_if_missing=False)
    assert L.ngb_create(None, None) == -1
    assert b"NULL" in L.ngb_last_error(None)
    h = ctypes.c_void_p()
    cfg = ngb.SimConfig(0.0, 1, 0, 0, None, 0, 1, 0, 0, 0)  # dt = 0 is rejected before any CUDA call
    assert L.ngb_create(ctypes.byref(h), ctypes.byref(cfg)) == -1
    assert L.ngb_destroy(None) == 0
