"""Textual variants of the FP64 oracle, compiled into a temporary directory.

TEST INFRASTRUCTURE ONLY.  Two uses:
  - mutation checks of the oracle's pins: a plausible mistake is planted in a
    copy of ``ccfr_oracle.c`` (a sort order flipped, the retraction moved, a
    pass dropped) and the pins must notice it;
  - studies of the readings of the paper (the halting study compares the
    retraction after every Alg. 1 call with one retraction per pass).

A variant is the oracle source with a list of (old, new) snippet
replacements; each snippet must occur exactly once, so a variant that no
longer applies fails loudly instead of silently testing the unmodified
oracle.  The variant is loaded through a fresh instance of ``oracle.py``
whose library path points at the variant's build.
"""
from __future__ import annotations

import hashlib
import importlib.util
import tempfile
from pathlib import Path

_HERE = Path(__file__).resolve().parent
_ROOT = Path(tempfile.gettempdir()) / "ccfr_oracle_variants"


def apply(replacements) -> str:
    """The oracle source with each (old, new) replacement applied once."""
    src = (_HERE / "ccfr_oracle.c").read_text()
    for old, new in replacements:
        n = src.count(old)
        if n != 1:
            raise ValueError(f"variant snippet found {n} times (need exactly 1): {old[:80]!r}")
        src = src.replace(old, new)
    return src


def load(name: str, replacements):
    """A module with the API of ``oracle.oracle`` backed by the variant."""
    src = apply(replacements)
    tag = hashlib.sha1(src.encode()).hexdigest()[:12]
    d = _ROOT / f"{name}_{tag}"
    d.mkdir(parents=True, exist_ok=True)
    c_file = d / "ccfr_oracle.c"
    if not c_file.exists() or c_file.read_text() != src:
        c_file.write_text(src)
    spec = importlib.util.spec_from_file_location(f"oracle_variant_{name}_{tag}", _HERE / "oracle.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    # share the ctypes structures with the main module, so that parameter
    # blocks made by either module are accepted by the variant's functions
    from oracle import oracle as main
    mod.OrcParams, mod.OrcExtra, mod.OrcStepInfo = main.OrcParams, main.OrcExtra, main.OrcStepInfo
    mod._SRC = c_file
    mod._LIB = d / "_build" / "libccfr_oracle.so"
    mod._lib = None
    mod.lib()
    return mod
