"""The C-ABI library builds, loads and exports every entry point that
include/dsmc.h declares; the ctypes mirrors have the header's layout; and
argument validation answers without touching a GPU (CPU tests)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_cs_9902024_gb300 import build as B
from paper_cs_9902024_gb300 import dsmc as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dsmc.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dsmc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.check_output(["nm", "-D", "--defined-only", B.LIB_PATH]).decode()
    exported = set(re.findall(r" T (dsmc_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert sorted(D.EXPORTS) == names
    for n in names:
        getattr(lib, n)


def test_ctypes_layout_matches_header():
    prog = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "dsmc.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu\n", sizeof(dsmc_domain), sizeof(dsmc_cells),
             sizeof(dsmc_gas), sizeof(dsmc_boundary), sizeof(dsmc_options), sizeof(dsmc_stats));
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", offsetof(dsmc_boundary, n),
             offsetof(dsmc_options, stream), offsetof(dsmc_options, profile),
             offsetof(dsmc_options, autotune), offsetof(dsmc_options, shape),
             offsetof(dsmc_stats, ms_steps), offsetof(dsmc_stats, launches_kernel),
             offsetof(dsmc_stats, shape), offsetof(dsmc_options, checks),
             offsetof(dsmc_options, tune_cache), offsetof(dsmc_gas, partner),
             offsetof(dsmc_gas, n_sub));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-std=c99", "-I" + os.path.join(ROOT, "include"), src, "-o", exe])
        lines = subprocess.check_output([exe]).decode().split("\n")
    sizes = [int(x) for x in lines[0].split()]
    assert sizes == [C.sizeof(D.Domain), C.sizeof(D.Cells), C.sizeof(D.Gas),
                     C.sizeof(D.Boundary), C.sizeof(D.Options), C.sizeof(D.Stats)]
    offs = [int(x) for x in lines[1].split()]
    assert offs == [D.Boundary.n.offset, D.Options.stream.offset, D.Options.profile.offset,
                    D.Options.autotune.offset, D.Options.shape.offset,
                    D.Stats.ms_steps.offset, D.Stats.launches_kernel.offset, D.Stats.shape.offset,
                    D.Options.checks.offset, D.Options.tune_cache.offset,
                    D.Gas.partner.offset, D.Gas.n_sub.offset]


def _args():
    from paper_cs_9902024_gb300 import workloads as W
    return D._structs(W.duct64x32_n8())


def test_invalid_arguments_rejected_without_gpu(lib):
    dom, cells, gas, arr, nb = _args()
    h = C.c_void_p()
    opt = D.Options(struct_size=C.sizeof(D.Options))
    # null output handle, null structs, wrong struct sizes, bad geometry
    assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(gas), arr, nb, C.byref(opt),
                           None) == D.E_INVALID
    assert lib.dsmc_create(None, C.byref(cells), C.byref(gas), arr, nb, C.byref(opt),
                           C.byref(h)) == D.E_INVALID
    bad = D.Domain.from_buffer_copy(dom)
    bad.struct_size = 4
    assert lib.dsmc_create(C.byref(bad), C.byref(cells), C.byref(gas), arr, nb, C.byref(opt),
                           C.byref(h)) == D.E_INVALID
    bad = D.Domain.from_buffer_copy(dom)
    bad.dim = 4
    assert lib.dsmc_create(C.byref(bad), C.byref(cells), C.byref(gas), arr, nb, C.byref(opt),
                           C.byref(h)) == D.E_INVALID
    badc = D.Cells.from_buffer_copy(cells)
    badc.n[0] = 0
    assert lib.dsmc_create(C.byref(dom), C.byref(badc), C.byref(gas), arr, nb, C.byref(opt),
                           C.byref(h)) == D.E_INVALID
    badg = D.Gas.from_buffer_copy(gas)
    badg.omega = 1.5
    assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(badg), arr, nb, C.byref(opt),
                           C.byref(h)) == D.E_INVALID
    # collision-partner choice out of range; subcells per axis out of range
    for partner, n_sub in ((3, 1), (-1, 1), (1, 0), (1, 65)):
        badg = D.Gas.from_buffer_copy(gas)
        badg.partner, badg.n_sub = partner, n_sub
        assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(badg), arr, nb,
                               C.byref(opt), C.byref(h)) == D.E_INVALID
    # a gas struct that ends before the partner fields is still accepted as
    # far as the argument checks go (uniform choice); one shorter is not
    badg = D.Gas.from_buffer_copy(gas)
    badg.struct_size = D.Gas.partner.offset - 8
    assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(badg), arr, nb, C.byref(opt),
                           C.byref(h)) == D.E_INVALID
    badb = (D.Boundary * 1).from_buffer_copy(arr)
    badb[0].face = 5          # z face in 2-D
    assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(gas), badb, 1, C.byref(opt),
                           C.byref(h)) == D.E_INVALID
    assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(gas), arr, 33, C.byref(opt),
                           C.byref(h)) == D.E_INVALID
    # launch-shape entries out of range
    for i, v in ((0, -1), (1, 1 << 21), (2, 255), (2, 16385), (3, -5)):
        bo = D.Options.from_buffer_copy(opt)
        bo.shape[i] = v
        assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(gas), arr, nb, C.byref(bo),
                               C.byref(h)) == D.E_INVALID
    assert not h.value
    # calls on a null context fail cleanly
    assert lib.dsmc_run_ensemble(None, 1, 1e-6, 1, None, 0, 1) == D.E_INVALID
    assert lib.dsmc_get_samples(None, 0, 0, None, 0) == D.E_INVALID
    assert lib.dsmc_last_error(None)
    lib.dsmc_destroy(None)


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    dom, cells, gas, arr, nb = _args()
    h = C.c_void_p()
    opt = D.Options(struct_size=C.sizeof(D.Options))
    assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(gas), arr, nb, C.byref(opt),
                           C.byref(h)) == D.E_CUDA
    # an older caller's gas (no partner fields) and valid partner choices
    # pass the argument checks too
    short = D.Gas.from_buffer_copy(gas)
    short.struct_size = D.Gas.partner.offset
    short.partner = 7        # beyond the caller's struct: not read
    variants = [short]
    for partner, n_sub in ((1, 1), (1, 64), (2, 0)):
        g = D.Gas.from_buffer_copy(gas)
        g.partner, g.n_sub = partner, n_sub
        variants.append(g)
    for g in variants:
        assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(g), arr, nb, C.byref(opt),
                               C.byref(h)) == D.E_CUDA
    assert not h.value


def test_binding_refuses_to_run_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_cs_9902024_gb300 import workloads as W
    with pytest.raises(D.DsmcError):
        D.Ensemble(W.duct64x32_n8())
