"""Host side of the learned part (no GPU): the bound-margin calibration of the
library (progress_learned_margin, a host computation) and a check that the
Python binding of the learned part only marshals tensors -- every piece of its
arithmetic (labels, targets, predicted bounds, branch bits and their confident
prefix) runs in the library."""

import ast
import os

import torch

from paper_2401_13772_gb300 import learned as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_calibrated_margin_covers_the_overshoot_quantile():
    g = torch.Generator().manual_seed(0)
    T = torch.rand(1000, 2, generator=g) * 0.2
    over = torch.linspace(0.0, 0.1, 1000)
    Y = T.clone()
    Y[:, 0] += over          # predictions above the target by 0 .. 0.1
    Y[:, 1] -= 0.05          # under-shooting is harmless
    m = L.calibrate_margin(Y, T, quantile=0.97, floor=0.0)
    assert abs(m - 0.097) < 1e-3
    covered = (Y[:, 0] - m <= T[:, 0] + 1e-12).double().mean().item()
    assert covered >= 0.97
    assert L.calibrate_margin(T, T, floor=0.02) == 0.02
    # exact order statistics: quantile 1 is the largest overshoot, 0 the smallest
    assert abs(L.calibrate_margin(Y, T, quantile=1.0, floor=0.0) - 0.1) < 1e-7
    assert L.calibrate_margin(Y, T, quantile=0.0, floor=0.0) == 0.0


# torch calls that only allocate, move or reshape memory
ALLOC = {"empty", "zeros", "empty_like", "zeros_like", "from_numpy", "randperm", "Generator",
         "full"}
# tensor methods that only move memory or read metadata
MOVE = {"to", "contiguous", "cpu", "numpy", "data_ptr", "numel", "clone", "manual_seed",
        "cuda_stream", "current_stream"}
# host-side functions allowed to compute with plain numbers (sizes, the
# parameter initialisation drawn with numpy, the mini-batch loop and its loss log)
HOST_MATH_OK = {"__init__", "fit"}


# integer sizes and counters (shapes, output widths, the Adam step count)
SIZE_NAMES = {"kmax", "step", "N_BOUNDS", "N_FEAT"}


def is_size(x):
    if isinstance(x, ast.Constant):
        return True
    if isinstance(x, ast.Name):
        return x.id in SIZE_NAMES
    if isinstance(x, ast.Attribute):
        return x.attr in SIZE_NAMES
    if isinstance(x, ast.Subscript):
        return isinstance(x.value, ast.Attribute) and x.value.attr == "shape"
    return False


def test_learned_binding_only_marshals():
    src = open(os.path.join(ROOT, "paper_2401_13772_gb300", "learned.py")).read()
    tree = ast.parse(src)
    bad = []

    def visit(node, func):
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            func = node.name
        if isinstance(node, (ast.BinOp, ast.AugAssign, ast.UnaryOp, ast.Compare)):
            if isinstance(node, ast.BinOp):
                ok_num = all(is_size(x) for x in (node.left, node.right))
            elif isinstance(node, ast.AugAssign):
                ok_num = is_size(node.target) and is_size(node.value)
            else:
                ok_num = False
            ok_none = isinstance(node, ast.Compare) and any(
                isinstance(c, ast.Constant) and c.value is None for c in node.comparators)
            ok_not = isinstance(node, ast.UnaryOp) and isinstance(node.op, ast.Not)
            if func not in HOST_MATH_OK and not (ok_num or ok_none or ok_not):
                bad.append((func, node.lineno, ast.unparse(node)))
        if isinstance(node, ast.Call) and isinstance(node.func, ast.Attribute):
            base = node.func.value
            name = node.func.attr
            if isinstance(base, ast.Name) and base.id == "torch" and name not in ALLOC:
                bad.append((func, node.lineno, ast.unparse(node)))
        for ch in ast.iter_child_nodes(node):
            visit(ch, func)

    visit(tree, "<module>")
    assert not bad, bad
