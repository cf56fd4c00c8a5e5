"""Each plausible misreading of Appendix A's error norm and controller, planted in a copy of the
oracle, fails one of the pins of tests/test_oracle_controller.py (CPU only).

The copies are compiled from the oracle's sources with one textual change each, into a temporary
directory; the pins then run on the mutant library in place of the oracle's own. A mutation that
no pin catches would be a reading on which the oracle and the GPU path could agree while both
being wrong.
"""
import concurrent.futures as cf
import ctypes
import os
import shutil

import pytest

import oracle as O
from oracle import build as obuild
from test_oracle_controller import check_linear, check_scipy_rk45

SRC = os.path.dirname(os.path.abspath(O.__file__))

# (name, original text, planted text): each original must occur exactly once in oracle.cpp
MUTANTS = [
    ("scale on |y| alone", "double sc = atol + rtol * (a > b ? a : b);", "double sc = atol + rtol * a;"),
    ("scale on |y+| alone", "double sc = atol + rtol * (a > b ? a : b);", "double sc = atol + rtol * b;"),
    ("exponent -1/(nu+1)", "o.beta1 : 1.0 / nu;", "o.beta1 : 1.0 / (nu + 1);"),
    ("norm without the mean over components", "err = std::sqrt(sq / d);", "err = std::sqrt(sq);"),
    ("no safety factor after accepts", "double fac = o.safety * std::pow(err, -beta1)",
     "double fac = 1.0 * std::pow(err, -beta1)"),
    ("halving after every reject", "\n        fac = o.safety * std::pow(err, -beta1)",
     "\n        fac = 0.5 + 0.0 * std::pow(err, -beta1)"),
    ("no floor after rejects", "        if (fac < o.alpha_min) fac = o.alpha_min;\n      }\n      h = h * fac;",
     "      }\n      h = h * fac;"),
    ("err_prev kept across a reject", "      h = h * fac;\n      err_prev = 1.0;", "      h = h * fac;"),
    ("err_prev not floored at 1e-4", "err_prev = err > 1e-4 ? err : 1e-4;", "err_prev = err;"),
]


def _build_mutant(tmp, i, orig, new):
    d = os.path.join(tmp, "m%d" % i)
    os.makedirs(d)
    for f in obuild.SOURCES + obuild.HEADERS:
        shutil.copy(os.path.join(SRC, f), d)
    path = os.path.join(d, "oracle.cpp")
    src = open(path).read()
    assert src.count(orig) == 1, (i, orig, src.count(orig))
    open(path, "w").write(src.replace(orig, new))
    return obuild.compile_lib(d, os.path.join(d, "liboracle.so"))


def _pins_fail():
    """True if at least one pin fails on the library currently loaded as the oracle."""
    for check in (check_scipy_rk45, check_linear):
        try:
            check()
        except AssertionError:
            return True
    return False


def _caught_with(lib):
    saved = O._lib
    O._lib = lib
    try:
        return _pins_fail()
    finally:
        O._lib = saved


def test_pins_pass_on_the_oracle():
    assert not _pins_fail()


def test_every_planted_misreading_fails_a_pin(tmp_path):
    with cf.ThreadPoolExecutor(min(len(MUTANTS), os.cpu_count() or 4)) as ex:
        libs = list(ex.map(lambda a: _build_mutant(str(tmp_path), a[0], a[1][1], a[1][2]), enumerate(MUTANTS)))
    missed = [name for (name, _, _), path in zip(MUTANTS, libs) if not _caught_with(ctypes.CDLL(path))]
    assert not missed, missed


def test_paper_ceiling_is_pinned(monkeypatch):
    """The oracle's default ceiling alpha_max = 5 (Eq. controller): a default of 10 fails the
    closed-form pin, which runs with the default options."""
    d = list(O.opts.__defaults__)
    names = O.opts.__code__.co_varnames[: O.opts.__code__.co_argcount]
    d[names.index("alpha_max") - (len(names) - len(d))] = 10.0
    monkeypatch.setattr(O.opts, "__defaults__", tuple(d))
    with pytest.raises(AssertionError):
        check_linear()
