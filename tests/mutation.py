"""Planting a mistake in one oracle function and running the pins against it (CPU only).

A mutant is the oracle function's own source with one textual replacement (a dropped term,
a flipped sign, a transposed operand, a wrong index), compiled in a copy of its module's
namespace. Every reference to the original function inside the ``oracle`` package is then
patched (pytest's ``monkeypatch``, undone after the test), so callers elsewhere in the
oracle pick the mutant up. ``failing_pins`` runs the plain pin tests of a test module,
expanding their ``parametrize`` marks, and returns the cases that fail.
"""
import inspect
import itertools
import sys
import textwrap
import warnings

import numpy as np
import pytest


def plant(monkeypatch, module, fname, old, new):
    """Replace ``old`` (which must occur exactly once) by ``new`` in ``module.fname``."""
    orig = getattr(module, fname)
    src = textwrap.dedent(inspect.getsource(orig))
    if src.count(old) != 1:
        raise ValueError(f"{fname}: {old!r} occurs {src.count(old)} times")
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant of {fname}>", "exec"), ns)
    mutant = ns[fname]
    for name, mod in list(sys.modules.items()):
        if mod is None or not (name == "oracle" or name.startswith("oracle.")):
            continue
        for attr, val in list(vars(mod).items()):
            if val is orig:
                monkeypatch.setattr(mod, attr, mutant)
    return mutant


def _cases(fn):
    """(label, kwargs) for every combination of a test function's parametrize marks."""
    axes = []
    for m in getattr(fn, "pytestmark", []):
        if m.name != "parametrize":
            continue
        names = m.args[0]
        names = [s.strip() for s in names.split(",")] if isinstance(names, str) else list(names)
        axes.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in m.args[1]])
    for combo in itertools.product(*axes):
        kw = {}
        for part in combo:
            kw.update(part)
        yield fn.__name__ + (str(sorted(kw.items())) if kw else ""), kw


def pin_cases(test_module):
    """Every plain pin of a test module: test functions whose arguments are all parametrized."""
    out = []
    for name, fn in vars(test_module).items():
        if not (name.startswith("test_") and callable(fn)) or "planted" in name:
            continue
        params = set(inspect.signature(fn).parameters)
        for label, kw in _cases(fn):
            if params <= set(kw):
                out.append((label, fn, kw))
    return out


def failing_pins(cases, skipped=None):
    """(label, exception type) of every pin case that fails.

    A pin that raises (an assertion, or an error such as an index out of range) counts as
    failing; the unmutated oracle passes every pin, so the mutant is what made it fail. A pin
    that skips itself (an optional package missing) is listed in ``skipped`` if given.
    """
    failed = []
    with _quiet():
        for label, fn, kw in cases:
            try:
                fn(**kw)
            except pytest.skip.Exception:
                if skipped is not None:
                    skipped.append(label)
            except Exception as e:  # noqa: BLE001 - any failure of a pin counts
                failed.append((label, type(e).__name__))
    return failed


class _quiet:
    """Silence numpy's floating-point warnings while mutants run (overflow, 0/0)."""

    def __enter__(self):
        self._np = np.seterr(all="ignore")
        self._w = warnings.catch_warnings()
        self._w.__enter__()
        warnings.simplefilter("ignore")

    def __exit__(self, *exc):
        np.seterr(**self._np)
        return self._w.__exit__(*exc)
