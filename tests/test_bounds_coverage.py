"""Source checks that keep the bounds-checked build complete (CPU): every
read of a walker-level index array in the kernels (the processing order
and the parents) passes through bounded(), and every trace write uses the
checked slot. An edit that adds an unchecked read fails here before it
reaches a GPU."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KERNELS = os.path.join(ROOT, "paper_1909_01589_gb300", "csrc", "lrdmc_kernels.cu")


def _code_lines():
    out = []
    for no, line in enumerate(open(KERNELS), 1):
        code = line.split("//")[0]
        if code.strip():
            out.append((no, code))
    return out


def _is_write(code, m):
    """The indexed element is assigned (the access is a store)."""
    depth, i = 0, m.end() - 1
    while i < len(code):
        depth += code[i] == "["
        depth -= code[i] == "]"
        i += 1
        if depth == 0:
            break
    return re.match(r"\s*=[^=]", code[i:]) is not None


def test_walker_index_reads_are_bounded():
    reads = 0
    for no, code in _code_lines():
        for m in re.finditer(r"P\.(order|parent)\[", code):
            if _is_write(code, m):
                continue
            reads += 1
            before = code[:m.start()]
            assert before.rstrip().endswith("bounded("), f"line {no}: unchecked read of P.{m.group(1)}: {code.strip()}"
    assert reads >= 4  # order and parent in both interval kernels


def test_trace_writes_use_the_checked_slot():
    writes = 0
    for no, code in _code_lines():
        for m in re.finditer(r"P\.trace\[([^\]]*)\]", code):
            writes += 1
            assert re.search(r"\bkt\b", m.group(1)), f"line {no}: trace slot not checked: {code.strip()}"
    assert writes == 4
    src = open(KERNELS).read()
    assert "const uint64_t kt = bounded(k, P.trace_cap, P.err);" in src


def test_bounded_is_identity_without_the_macro():
    text = open(os.path.join(ROOT, "paper_1909_01589_gb300", "csrc", "lrdmc_internal.h")).read()
    body = text[text.index("__device__ __forceinline__ I bounded"):]
    body = body[:body.index("\n}\n")]
    assert "#ifdef LRDMC_BOUNDS" in body and "return I(0);" in body
    # outside the #ifdef the function returns its argument
    tail = body[body.index("#endif"):]
    assert "return i;" in tail
