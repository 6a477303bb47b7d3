import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built engine")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def program_from_spec(spec):
    """Program object from a golden-fixture program spec."""
    from paper_2011_08373_gb300.synth import make_program

    stmts = []
    for st in spec["stmts"]:
        d = dict(st)
        if "guard" in d:
            d["guard"] = tuple(d["guard"])
        stmts.append(d)
    return make_program(
        stmts, blocks=spec["blocks"], threads=spec["threads"],
        m_shared=spec.get("m_shared", 0), m_global=spec.get("m_global", 0),
        slot_level=spec["slot_level"], slot_guard=[tuple(g) for g in spec["slot_guard"]],
        slot_weight=spec["slot_weight"], existing_mask=spec["existing_mask"],
        perms=[np.array(t, np.uint32) for t in spec.get("perms", [])],
        loops=[tuple(l) for l in spec.get("loops", [])], neg_clauses=spec.get("neg_clauses", []),
        slot_pos=spec.get("slot_pos"))
