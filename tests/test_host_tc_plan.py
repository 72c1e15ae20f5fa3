"""Host logic of the grouped tensor-core launch (no GPU): the work-item table,
the sign / power-of-two segment weights of merged contractions, and the alpha
merge classes, through the inline helpers of tcgemm.h compiled with g++."""
import bisect
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2511_03567_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    exe = str(tmp_path_factory.mktemp("tcplan") / "tc_plan_driver")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", cuda_inc,
                    os.path.join(HERE, "host", "tc_plan_driver.cpp"), "-o", exe], check=True)

    def run(text):
        r = subprocess.run([exe], input=text, capture_output=True, text=True, check=True)
        return r.stdout.split("\n")
    return run


def _plan(rng, n_ops, k_max):
    """Random ops (some merged from several K segments) grouped into clusters
    the way the builder does: single-pair ops share a cluster per A operand,
    every merged op is a cluster of its own."""
    ops, segs, clusters = [], [], []
    i = 0
    while i < n_ops:
        nseg = int(rng.integers(2, 6)) if rng.random() < 0.4 else 1
        if nseg > 1:
            lens = [int(x) for x in rng.integers(1, 30, size=nseg)]
            ops.append(dict(nt=int(rng.integers(1, 4)), nseg=nseg, seg0=len(segs), kt0=lens[0]))
            segs += lens[1:]
            members, kt_total = [len(ops) - 1], sum(lens)
            i += 1
        else:
            kt_total = int(rng.integers(1, 120))
            members = []
            for _ in range(int(rng.integers(1, 4))):
                ops.append(dict(nt=int(rng.integers(1, 4)), nseg=1, seg0=len(segs), kt0=kt_total))
                members.append(len(ops) - 1)
                i += 1
        ks = -(-kt_total // k_max)
        kps = -(-kt_total // ks)
        ksplit = -(-kt_total // kps)
        W = sum(ops[q]["nt"] for q in members)
        clusters.append(dict(op0=members[0], nops=len(members), mt=int(rng.integers(1, 4)),
                             kt_total=kt_total, kps=kps, ksplit=ksplit, W=W))
    begin = 0
    for c in clusters:
        c["begin"] = begin
        begin += c["mt"] * c["ksplit"] * c["W"]
    return ops, segs, clusters, begin


def _expected(ops, segs, clusters):
    out = []
    for c in clusters:
        for u in range(c["mt"] * c["ksplit"]):
            mi, ks = divmod(u, c["ksplit"])
            kt0 = ks * c["kps"]
            kt1 = min(c["kt_total"], kt0 + c["kps"])
            for q in range(c["op0"], c["op0"] + c["nops"]):
                o = ops[q]
                lens = [o["kt0"]] + segs[o["seg0"]:o["seg0"] + o["nseg"] - 1]
                ends = list(np.cumsum(lens))
                s0 = bisect.bisect_right(ends, kt0)
                s1 = bisect.bisect_right(ends, kt1 - 1)
                for ni in range(o["nt"]):
                    out.append((q, mi, ni, kt0, kt1, s0, s1, int(ends[s0])))
    return out


def _items_text(ops, segs, clusters):
    lines = ["items", str(len(clusters))]
    lines += [" ".join(str(c[k]) for k in ("begin", "op0", "nops", "mt", "kt_total", "kps", "ksplit", "W"))
              for c in clusters]
    lines.append(str(len(ops)))
    lines += ["%d %d %d %d" % (o["nt"], o["nseg"], o["seg0"], o["kt0"]) for o in ops]
    lines.append(str(len(segs)))
    lines += [str(x) for x in segs]
    return "\n".join(lines) + "\n"


@pytest.mark.parametrize("seed,k_max", [(0, 43), (1, 7), (2, 1), (3, 200)])
def test_item_table_matches_enumeration(driver, seed, k_max):
    rng = np.random.default_rng(seed)
    ops, segs, clusters, total = _plan(rng, 25, k_max)
    out = driver(_items_text(ops, segs, clusters))
    assert out[0] == "ok %d" % total
    got = [tuple(int(x) for x in line.split()) for line in out[1:1 + total]]
    assert got == _expected(ops, segs, clusters)
    # every (op, m tile, n tile) covers the op's whole K range once, in order
    cover = {}
    for q, mi, ni, kt0, kt1, s0, s1, send in got:
        cover.setdefault((q, mi, ni), []).append((kt0, kt1))
    for (q, mi, ni), r in cover.items():
        o = ops[q]
        ktot = o["kt0"] + sum(segs[o["seg0"]:o["seg0"] + o["nseg"] - 1])
        assert r[0][0] == 0 and r[-1][1] == ktot
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))


def test_item_table_rejects_16_bit_overflow(driver):
    ops = [dict(nt=1, nseg=1, seg0=0, kt0=70000)]
    clusters = [dict(begin=0, op0=0, nops=1, mt=1, kt_total=70000, kps=70000, ksplit=1, W=1)]
    assert driver(_items_text(ops, [], clusters))[0] == "overflow"


def test_segment_weights_reproduce_alphas(driver):
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = int(rng.integers(1, 9))
        e0 = int(rng.integers(-6, 3))
        es = sorted(int(x) for x in rng.integers(e0, e0 + 16, size=n))
        es[0] = e0
        es.sort()
        signs = rng.choice([-1.0, 1.0], size=n)
        alphas = [float(sg * 2.0 ** e) for sg, e in zip(signs, es)]
        out = driver("weights %d %s\n" % (n, " ".join(repr(a) for a in alphas)))[0].split()
        assert out[0] == "ok", alphas
        base = float(out[1])
        codes = [int(x) for x in out[2:]]
        for a, c in zip(alphas, codes):
            assert (-1.0 if c & 1 else 1.0) * base * 2.0 ** (c >> 1) == a
            assert (c >> 1) <= 15


@pytest.mark.parametrize("alphas", [[1.0, 3.0], [2.0, 1.0], [1.0, 65536.0], [0.0, 1.0], [0.5, -0.25]])
def test_segment_weights_reject_other_forms(driver, alphas):
    out = driver("weights %d %s\n" % (len(alphas), " ".join(repr(a) for a in alphas)))[0]
    assert out == "bad"


def test_alpha_merge_classes(driver):
    def key(a):
        return driver("class %r\n" % a)[0]
    window = {key(s * 2.0 ** e) for e in range(-8, 8) for s in (-1.0, 1.0)}
    assert len(window) == 1  # +-2^-8 .. +-2^7 merge: sign and exponent go into the MMA
    assert key(2.0 ** 8) not in window and key(2.0 ** -9) not in window
    assert key(2.0 ** 8) == key(2.0 ** 23)
    assert key(3.0) != key(-3.0) and key(3.0) not in window and key(0.75) not in window
    assert key(3.0) == key(3.0)
