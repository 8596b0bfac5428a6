import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def read_golden_cases(name):
    """Parses tests/golden/<name> into a list of dicts."""
    cases, cur = [], None
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            key, *rest = line.split()
            if key == "case":
                cur = {"name": rest[0], "bfs": []}
            elif key == "end":
                cases.append(cur)
                cur = None
            elif key == "n":
                cur["n"] = int(rest[0])
            elif key == "n_plus":
                cur["n_plus"] = int(rest[0])
            elif key == "edges":
                pairs = [tuple(int(x) for x in e.split("-")) for e in rest]
                cur["src"] = [p[0] for p in pairs]
                cur["dst"] = [p[1] for p in pairs]
            elif key == "P":
                cur["P"] = [int(x) for x in rest]
            elif key == "bfs":
                cur["bfs"].append((int(rest[0]), [int(x) for x in rest[1:]]))
    return cases
