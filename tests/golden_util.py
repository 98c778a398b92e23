"""Reader for the closed-form text fixtures under tests/golden/."""
import math
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def expr(s):
    return float(eval(s, {"__builtins__": {}}, {"sqrt": math.sqrt, "pi": math.pi}))


def rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            out.append(line.split())
    return out
