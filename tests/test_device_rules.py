"""Rules the CUDA sources keep so that no kernel can trap or wait forever (CPU only, a scan).

* No ``__trap``, ``trap`` instruction or device ``assert``: device-detected conditions are
  counted in the caller's status words instead.
* The raw ``mbarrier.try_wait`` instruction appears only in the shared wait helpers, and every
  function that polls it (``mbar_try_wait``) or a counter in global memory (``ld_acquire``) does
  so in a loop with an iteration limit.
* No ``while (true)`` / ``while (1)``; a ``for (;;)`` appears only as a work loop whose body
  makes its waits through those bounded helpers and leaves by ``break``.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1707_02162_gb300", "csrc")

BOUNDED_HELPERS = ("mbar_wait_bounded", "mbar_wait_bounded_n", "wait_bar", "wait_count")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            out[f] = open(os.path.join(CSRC, f)).read()
    return out


def _strip_comments(text):
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def _block(text, open_pos):
    """Text of the brace-matched block whose '{' is at open_pos."""
    depth = 0
    for i in range(open_pos, len(text)):
        if text[i] == "{":
            depth += 1
        elif text[i] == "}":
            depth -= 1
            if depth == 0:
                return text[open_pos:i + 1]
    raise AssertionError("unbalanced braces")


def _enclosing_function(text, pos):
    """Name of the last function definition that starts before pos."""
    defs = list(re.finditer(r"\b(\w+)\s*\([^;{]*\)\s*(?:const\s*)?\{", text[:pos]))
    names = [m.group(1) for m in defs if m.group(1) not in ("if", "for", "while", "switch")]
    return names[-1] if names else None


def test_no_traps_or_device_asserts():
    srcs = _sources()
    assert srcs
    for f, text in srcs.items():
        code = _strip_comments(text)
        assert "__trap" not in code, f
        assert not re.search(r'asm[^;]*"\s*trap', code), f
        assert not re.search(r"(?<!static_)\bassert\s*\(", code), f


def test_raw_mbarrier_wait_only_in_the_helpers():
    for f, text in _sources().items():
        if "mbarrier.try_wait" in _strip_comments(text):
            assert f == "device_sync.cuh", f


def test_every_poll_sits_in_a_bounded_loop():
    found = set()
    for f, text in _sources().items():
        code = _strip_comments(text)
        for m in re.finditer(r"\b(mbar_try_wait|ld_acquire)\s*\(", code):
            line = code[code.rfind("\n", 0, m.start()) + 1:m.start()]
            if "__device__" in line:
                continue                                   # the definitions themselves
            fn = _enclosing_function(code, m.start())
            found.add(fn)
            assert fn in BOUNDED_HELPERS, f"{f}: {m.group(1)} polled in {fn}"
            start = code.rfind(fn, 0, m.start())
            body = _block(code, code.index("{", start))
            assert re.search(r"for\s*\(\s*uint32_t\s+i\s*=\s*0\s*;\s*i\s*<\s*\w+\s*;", body), f"{f}: {fn}"
    assert found, "no polling helper found"


def test_no_unbounded_loop_forms():
    for f, text in _sources().items():
        code = _strip_comments(text)
        assert not re.search(r"while\s*\(\s*(true|1)\s*\)", code), f
        for m in re.finditer(r"for\s*\(\s*;\s*;\s*\)\s*\{", code):
            body = _block(code, m.end() - 1)
            assert "break" in body, f"{f}: for (;;) without a break"
            assert any(h + "(" in body for h in BOUNDED_HELPERS) or "atomicAdd" in body, \
                f"{f}: for (;;) whose waits are not the bounded helpers"
