"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/*.h declares (no compute call: this runs without a GPU)."""
import glob
import os
import re

from paper_2606_09799_gb300 import build as libbuild
from paper_2606_09799_gb300 import ibm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ibm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = ibm.load()
    names = declared_symbols()
    assert {"ibm_create_grid", "ibm_set_surface", "ibm_step", "ibm_get_fields"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(ibm.EXPORTS) <= names


def test_library_is_built_for_sm_103a_in_tree():
    path = libbuild.build()
    assert path.startswith(os.path.join(ROOT, "paper_2606_09799_gb300"))
    assert "arch=compute_103a,code=sm_103a" in " ".join(libbuild.ARCH)
    assert ibm.ibm_version().startswith("ibm-gb300")


def test_bad_arguments_are_rejected_without_a_gpu():
    L = ibm.load()
    import ctypes
    h = ctypes.c_void_p()
    for bad in (ibm.ibm_grid_desc(14, 64, 64, 1, 1, 1, 100, 1e-3, 0, 0, 0, 1),     # 14 = 2 * 7
                ibm.ibm_grid_desc(64, 2, 64, 1, 1, 1, 100, 1e-3, 0, 0, 0, 1),      # ny too small
                ibm.ibm_grid_desc(64, 64, 64, 1, 1, 1, -1, 1e-3, 0, 0, 0, 1),      # Re <= 0
                ibm.ibm_grid_desc(64, 64, 64, 1, 1, 1, 100, 1e-3, 7, 0, 0, 1)):    # unknown scheme
        assert L.ibm_create_grid(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    assert L.ibm_create_grid(None, None, ctypes.byref(h)) == 1
    assert L.ibm_destroy(None) == 1
