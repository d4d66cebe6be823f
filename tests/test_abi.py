"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/dfscf.h declares (no GPU needed; nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^(?:const\s+)?\w+[\s\*]+(\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_core_entry_points():
    names = declared_functions()
    for required in ("df_metric_chol", "df_build_B", "df_jk", "scf_run", "df_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2506_06661_gb300 as dfscf
    path = dfscf._build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_size_queries_without_gpu():
    import paper_2506_06661_gb300 as dfscf
    L = dfscf.lib()
    assert L.df_B_ld(100) == 5056  # 5050 rounded up to 32
    assert L.df_nao_pad(100) == 128
    assert L.df_B_bytes(100, 300, 0) == 300 * 5056 * 8
    assert L.df_B_bytes(100, 300, 2) == 0
    assert L.df_jk_work_bytes(100, 300, 10, 0) > 0
    assert L.scf_work_bytes(100, 300, 10, 0) > L.df_B_bytes(100, 300, 0)


def test_argument_errors_are_host_side():
    import paper_2506_06661_gb300 as dfscf
    L = dfscf.lib()
    rc = L.df_jk(None, 100, 300, 0, None, None, 0, None, None, None, 0, None)
    assert rc == dfscf.DF_ERR_ARG
    assert b"df_jk" in L.df_last_error()
    rc = L.df_boys_f0(None, -1, None, None)
    assert rc == dfscf.DF_ERR_ARG


def test_tuning_knobs_host_side():
    import paper_2506_06661_gb300 as dfscf
    from paper_2506_06661_gb300 import tune
    L = dfscf.lib()
    assert L.df_tune_get(b"jpass2_rows") == 256
    assert L.df_tune_get(b"nope") == -1
    assert L.df_tune_set(b"jpass2_rows", 9999) == dfscf.DF_ERR_ARG
    w0 = L.df_jk_work_bytes(1500, 4500, 150, 0)
    tune.set_knob("jpass2_rows", 128)
    try:
        assert L.df_jk_work_bytes(1500, 4500, 150, 0) > w0   # more J slices, larger partial buffer
    finally:
        tune.set_knob("jpass2_rows", 256)
    assert tune.bucket(1500, 4500, 150, "mixed") == "mixed:nao2048:naux8192:nocc256"
    # df_tune_reset restores every knob's built-in value
    defaults = {k: L.df_tune_get(k.encode()) for k in ("syrk_split", "umma_max_stages", "stability")}
    tune.set_knob("syrk_split", 44)
    tune.set_knob("umma_max_stages", 2)
    tune.set_knob("stability", 2)
    tune.reset()
    assert {k: L.df_tune_get(k.encode()) for k in defaults} == defaults == {
        "syrk_split": 0, "umma_max_stages": 8, "stability": 0}


def test_header_is_plain_c_and_links():
    """include/dfscf.h is consumable from C99, and a C program calling the core entry points
    links against the built library (compiled from standard input, linked to /dev/null)."""
    import shutil
    import subprocess
    import paper_2506_06661_gb300 as dfscf
    gcc = shutil.which("gcc")
    if gcc is None:
        import pytest
        pytest.skip("gcc not available")
    lib_path = dfscf._build.build()
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(dfscf._build.nvcc()))), "include")
    prog = ("#include \"dfscf.h\"\n"
            "typedef void (*fn)(void);\n"
            "int main(void) {\n"
            "  volatile fn used[] = {(fn)df_metric_chol, (fn)df_build_B, (fn)df_jk, (fn)scf_run, (fn)scf_run_batch};\n"
            "  size_t b = df_B_bytes(100, 300, DF_FP64);\n"
            "  return (b > 0 && df_version() > 0 && df_last_error() != 0 && used[0] != 0) ? 0 : 1;\n"
            "}\n")
    cmd = [gcc, "-x", "c", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, "-",
           "-L", os.path.dirname(lib_path), "-l:" + os.path.basename(lib_path), "-o", os.devnull]
    r = subprocess.run(cmd, input=prog, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_host_tensors_are_refused_before_reaching_the_library():
    """The binding hands only contiguous CUDA tensors to the C ABI: a host tensor (or a
    non-contiguous one) raises TypeError instead of passing a host pointer to device code."""
    import torch
    import paper_2506_06661_gb300 as dfscf
    with pytest.raises(TypeError):
        dfscf._ptr(torch.zeros(4, dtype=torch.float64))
    with pytest.raises(TypeError):
        dfscf.default_opts(guess_params=torch.zeros(4, dtype=torch.float32))
    assert dfscf._ptr(None) is None
