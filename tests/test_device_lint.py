"""Static checks on the CUDA sources (no GPU needed).

A warp collective (__shfl*_sync, __ballot_sync, __all_sync, __any_sync,
__syncwarp) must be executed by every lane its mask names.  A collective on
the right of && / || / ?: is skipped by lanes where the left side decides
the result, which leaves the other lanes waiting: such code is rejected."""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2511_03655_gb300", "csrc")
COLLECTIVE = re.compile(r"__(shfl\w*|ballot|all|any|match\w*|reduce\w*)_sync\s*\(|__syncwarp\s*\(")


def statements_with_collectives():
    for fn in sorted(os.listdir(CSRC)):
        if not fn.endswith((".cu", ".cuh")):
            continue
        text = open(os.path.join(CSRC, fn)).read()
        text = re.sub(r"//[^\n]*", "", text)
        for m in COLLECTIVE.finditer(text):
            start = max(text.rfind(";", 0, m.start()), text.rfind("{", 0, m.start()),
                        text.rfind("}", 0, m.start())) + 1
            yield fn, text[start:m.start()], text.count("\n", 0, m.start()) + 1


def test_sources_found():
    assert any(True for _ in statements_with_collectives())


@pytest.mark.parametrize("fn,prefix,line", list(statements_with_collectives()))
def test_no_collective_behind_short_circuit(fn, prefix, line):
    assert not re.search(r"&&|\|\||\?", prefix), f"{fn}:{line}: collective after a short-circuit: {prefix.strip()}"
