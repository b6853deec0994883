"""The product path has no CPU fallback and never reaches the oracle.

* The package, the CUDA sources and the shared input generators import,
  include or load nothing under oracle/ (and the oracle nothing of theirs):
  the two sides share no code, so agreement between them is evidence.
* Without the built library the binding raises instead of computing
  anything else; host tensors are refused before any call into the library.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1803_09652_gb300")


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_and_generators_do_not_touch_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b|#\s*include\s*[<\"].*gbo)|libgbo|oracle/", re.M)
    tops = [(PKG, (".py", ".cu", ".cuh", ".h")), (os.path.join(ROOT, "synth"), (".py",)),
            (os.path.join(ROOT, "include"), (".h",))]
    hits = [f for top, ext in tops for f in _files(top, ext) if pat.search(open(f).read())]
    assert hits == []


def test_oracle_does_not_touch_the_product():
    src = open(os.path.join(ROOT, "oracle", "gbo.c")).read() + open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_1803_09652_gb300" not in src
    assert "gbremd" not in src
    assert not re.search(r"#\s*include\s*\"", src)          # only system headers


def test_missing_library_raises():
    import paper_1803_09652_gb300 as pkg
    with pytest.raises(RuntimeError, match="not built"):
        pkg.load(os.path.join(ROOT, "no_such_dir", "libgbremd.so"))


def test_host_tensors_are_refused():
    torch = pytest.importorskip("torch")
    import paper_1803_09652_gb300 as pkg
    with pytest.raises(ValueError, match="CUDA tensor"):
        pkg._ptr(torch.zeros(4))
