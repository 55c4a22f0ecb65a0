"""The C-ABI library builds, loads and exports every entry point that
include/nepzbl.h declares (no GPU needed)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nepzbl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("nep_init", "nep_compute", "md_step", "nep_free", "nep_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2305_08140_gb300 import nepzbl as N
    lib = N.load()
    out = subprocess.run(["nm", "-D", "--defined-only", N.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for n in _declared():
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(N.EXPORTED) <= exported


def test_struct_layouts_match_header():
    """ctypes mirrors of the ABI structs have the sizes a C compiler gives."""
    import ctypes as C
    import tempfile
    from paper_2305_08140_gb300 import nepzbl as N
    prog = ('#include <stdio.h>\n#include "nepzbl.h"\nint main(void){printf('
            '"%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(nep_params), sizeof(nep_md_state), '
            'sizeof(nep_stats), sizeof(nep_batch), sizeof(nep_targets), '
            'sizeof(nep_loss_weights), sizeof(nep_tune_table));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c])
        sizes = [int(v) for v in subprocess.check_output([exe]).split()]
    assert sizes == [C.sizeof(N.NepParams), C.sizeof(N.NepMdState), C.sizeof(N.NepStats),
                     C.sizeof(N.NepBatch), C.sizeof(N.NepTargets), C.sizeof(N.NepLossWeights),
                     C.sizeof(N.NepTuneTable)]


def test_init_without_gpu_fails_cleanly():
    """Without a usable GPU nep_init returns an error code instead of
    crashing (on a GPU machine it succeeds)."""
    import torch
    from paper_2305_08140_gb300 import inputs as I
    from paper_2305_08140_gb300 import nepzbl as N
    if torch.cuda.is_available():
        m = N.NEP(I.nep_model(1))
        m.close()
        return
    try:
        N.NEP(I.nep_model(1))
    except N.NepError as e:
        assert e.code == N.NEP_ERR_CUDA
    else:
        raise AssertionError("nep_init succeeded without a GPU")
