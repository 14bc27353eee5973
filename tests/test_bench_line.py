"""The benchmark's result line is strict JSON: values that are not finite (an
error bar over too few intervals) become null, numpy scalars become plain
numbers, and nothing else changes."""
import json
import math

import numpy as np

import bench


def test_result_line_is_strict_json():
    line = {"value": 2.5e7, "err": float("nan"), "inf": float("inf"), "ninf": -math.inf,
            "n": np.int64(60), "f": np.float32(0.5), "nested": {"a": [1.0, np.float64("nan"), "x"]},
            "flag": True, "none": None}
    text = bench.json_line(line)
    back = json.loads(text, parse_constant=lambda c: (_ for _ in ()).throw(ValueError(c)))
    assert back == {"value": 2.5e7, "err": None, "inf": None, "ninf": None, "n": 60, "f": 0.5,
                    "nested": {"a": [1.0, None, "x"]}, "flag": True, "none": None}
    assert "NaN" not in text and "Infinity" not in text
