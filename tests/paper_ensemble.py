"""The paper's rate-0.02 multi-edge ensemble (Sec. III-B), loaded from the
cited fixture tests/golden/met_ensemble_sec3b.json, in the (fraction,
degree vector) form the threshold tools take."""
import json
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "met_ensemble_sec3b.json")
with open(_PATH) as _f:
    FIXTURE = json.load(_f)


def _types(key):
    return [(num / den, tuple(t["degrees"])) for t in FIXTURE[key] for num, den in [t["fraction"]]]


PAPER_VN_PRINTED = _types("variable_types_printed")
PAPER_VN_BALANCED = _types("variable_types_read")
PAPER_CN = _types("check_types")
PAPER_THRESHOLD = FIXTURE["threshold_snr"]
PAPER_RATE = FIXTURE["rate"]
