"""Constants the paper prints (tests/golden/paper_constants.txt, each entry
with its passage) against what the library and the benchmark use.  Read as
text where importing would need the built library.  No GPU."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def golden():
    out = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_constants.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("=", 1))
            out[k] = v
    return out


def module_constants(path):
    tree = ast.parse(open(os.path.join(ROOT, path)).read())
    out = {}
    for node in tree.body:
        if isinstance(node, ast.Assign):
            try:
                val = ast.literal_eval(node.value)
            except ValueError:
                continue
            for t in node.targets:
                if isinstance(t, ast.Name):
                    out[t.id] = val
                elif isinstance(t, ast.Tuple) and isinstance(val, tuple):
                    for e, v in zip(t.elts, val):
                        out[e.id] = v
    return out


def test_block_plan_reads_as_the_paper_widths():
    """e/d blocks going down then up: the three pooled encoder blocks, the
    d96 block at the coarsest scale, the decoder blocks coming up (their
    widths by scale are the list reversed)."""
    from oracle import wnet as W
    from paper_2209_09965_gb300 import workloads as wl
    blocks = golden()["block_plan"].split("-")
    enc = tuple(int(b[1:]) for b in blocks if b[0] == "e")
    rest = [int(b[1:]) for b in blocks if b[0] == "d"]
    bot, dec_up = rest[0], rest[1:]
    cfg = (enc, bot, tuple(reversed(dec_up)))
    assert cfg == W.PAPER == wl.WNET_PAPER
    assert len(blocks) == 7 and len(enc) + 1 == 4 and len(dec_up) == 3   # the text counts 4 encoder, 3 decoder blocks


def test_loss_weights():
    g = golden()
    c = module_constants("paper_2209_09965_gb300/train.py")
    assert c["LAMBDA_S"] == float(g["lambda_s"]) and c["LAMBDA_T"] == float(g["lambda_t"])


def test_shadow_rate():
    from paper_2209_09965_gb300 import workloads as wl
    assert wl.MarchParams().shadow_rate == int(golden()["shadow_rate"])


def test_benchmark_runs_the_printed_settings():
    g = golden()
    settings = [tuple(float(x) for x in s.split()) for s in g["speedup_settings"].split(";")]
    src = open(os.path.join(ROOT, "bench.py")).read()
    m = re.search(r"for pb, sig in \(\((.*?)\)\):", src)
    assert m, "paper-settings loop not found"
    used = [tuple(float(x) for x in part.split(",")) for part in m.group(1).split("), (")]
    assert used == settings
    w, h = (int(x) for x in g["paper_frame"].split())
    assert re.search(rf"\b{w}\b", src) and re.search(rf"\b{h}\b", src)
