"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/rt3d.h declares (no compute calls: this runs without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rt3d_[a-z_]+)\s*\(", txt))
    return names


def test_header_declares_the_boundary():
    need = {"rt3d_create", "rt3d_destroy", "rt3d_set_cosmology", "rt3d_load_particles", "rt3d_trace",
            "rt3d_trace_device", "rt3d_trace_batch", "rt3d_histogram", "rt3d_status_string"}
    assert need <= declared()


def test_library_exports_every_declared_symbol():
    from paper_1110_4894_gb300 import build
    path = build.build()
    lib = C.CDLL(path)
    for name in sorted(declared()):
        assert hasattr(lib, name), name


def test_status_strings_and_no_device():
    import paper_1110_4894_gb300 as P
    L = P.lib()
    assert L.rt3d_status_string(0) == b"ok"
    assert L.rt3d_status_string(-6) == b"cosmology not set"
    assert L.rt3d_status_string(-99) == b"unknown status"
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        with pytest.raises(P.Rt3dError):
            P.Context(0)


def test_oracle_and_library_share_nothing():
    # the oracle and the CUDA path are separate programs: no file of one
    # includes, imports or links the other
    csrc = os.path.join(ROOT, "paper_1110_4894_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".cu", ".cuh", ".py", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt), f
                assert "orc.h" not in txt and "liborc" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h", ".py")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "rt3d" not in txt and "paper_1110_4894_gb300" not in txt, f


def declarations_with_comments():
    """(name, the comment block right above its declaration) for every
    entry point of include/*.h"""
    out = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        for m in re.finditer(r"^(?:int|const char \*)\s*(rt3d_[a-z_]+)\s*\(", txt, flags=re.M):
            head = txt[:m.start()]
            end = head.rfind("*/")
            start = head.rfind("/*", 0, end)
            between = head[end + 2:]
            # only #defines may sit between the comment and the declaration
            assert all(l.strip() == "" or l.startswith("#define") for l in between.splitlines()), m.group(1)
            out.append((m.group(1), head[start:end]))
    return out


def test_every_declaration_cites_its_passage():
    decl = declarations_with_comments()
    assert len(decl) == len(declared())
    cite = re.compile(r"\b(Sec\.|Eqs?\.|App\.|Fig\.)")
    for name, comment in decl:
        assert cite.search(comment) or "no counterpart" in comment, name
