"""Reader of tests/golden/paper_values.txt (values printed in the paper, with citations)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.txt")


def paper_values():
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (x.strip() for x in line.split("=", 1))
            out[k] = int(v) if v.isdigit() else float(v)
    return out
