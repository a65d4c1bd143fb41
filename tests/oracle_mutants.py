"""Planted-mistake copies of the oracle, for showing that a pin can fail.

``mutant(tmp_path, old, new)`` copies the oracle package into a temporary
folder with one source line of ``fpm_oracle.c`` replaced (the text ``old``
must occur exactly once), builds that copy with gcc and imports it under a
private module name.  The copy is used only on the CPU, by tests that assert
that a pin rejects the planted mistake; the oracle in the tree is untouched.
"""
from __future__ import annotations

import importlib.util
import itertools
import os
import shutil

import oracle

_count = itertools.count()


def mutant(tmp_path, old: str, new: str):
    src_dir = os.path.dirname(os.path.abspath(oracle.__file__))
    with open(os.path.join(src_dir, "fpm_oracle.c")) as f:
        src = f.read()
    if src.count(old) != 1:
        raise ValueError(f"planted mistake: {old!r} occurs {src.count(old)} times in the oracle")
    k = next(_count)
    d = tmp_path / f"oracle_mutant_{k}"
    d.mkdir()
    (d / "fpm_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(src_dir, "__init__.py"), d / "__init__.py")
    name = f"_oracle_mutant_{os.getpid()}_{k}"
    spec = importlib.util.spec_from_file_location(name, d / "__init__.py", submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod
