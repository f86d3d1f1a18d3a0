"""Planted mistakes for the oracle pins: a copy of an oracle function whose
source has one expression replaced, compiled in the function's own module
namespace, so that a test can check that its pins catch that slip."""
import inspect
import textwrap


def mutant(func, old, new):
    """``func`` with the source text ``old`` replaced by ``new`` (exactly once)."""
    src = textwrap.dedent(inspect.getsource(func))
    assert src.count(old) == 1, f"{old!r} must occur once in {func.__qualname__}"
    src = src.replace(old, new)
    ns = dict(func.__globals__)
    exec(compile(src, f"<mutant of {func.__qualname__}>", "exec"), ns)
    return ns[func.__name__]
