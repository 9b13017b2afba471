"""The device's branching helpers (csrc/bnb_common.cuh), run on the host.

The queue stores a sub-cube as integer cell coordinates and two levels; the
kernels decode them to FP64 geometry, pick the split (Sec. 4.1, reading R6)
and form the eight children.  The same __host__ __device__ functions are
compiled here into a host program with nvcc and checked against the
definition of the split written out in Python: a path of splits from the
root replayed in FP64 lands on the decoded cube, the eight children tile
their parent, the self-sum cache is dropped exactly on translation splits,
and the FP32 priority keys order like the floats they encode."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1812_01232_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include "bnb_common.cuh"
using namespace gosma;

static void put(const CubeGeom &g) {
    printf("%.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", g.r0[0], g.r0[1], g.r0[2], g.rhw,
           g.t0[0], g.t0[1], g.t0[2], g.thw[0], g.thw[1], g.thw[2]);
}

int main(int argc, char **argv) {
    if (!strcmp(argv[1], "keys")) {  // stdin: float bit patterns (hex); out: key, decoded bit pattern
        unsigned u;
        while (scanf("%x", &u) == 1) {
            float f;
            memcpy(&f, &u, 4);
            float b = key_value(order_key(f));
            unsigned v;
            memcpy(&v, &b, 4);
            printf("%u %x\n", order_key(f), v);
        }
        return 0;
    }
    if (!strcmp(argv[1], "rule")) {  // argv: lr lt psit -> 1 if the rotation is split
        Node n;
        memset(&n, 0, sizeof n);
        n.lr = (uint16_t)atoi(argv[2]);
        n.lt = (uint16_t)atoi(argv[3]);
        n.psit = (float)atof(argv[4]);
        printf("%d %.17g\n", (int)split_rotation(n), psi_r_level(n.lr));
        return 0;
    }
    // walk: stdin t_lo[3] t_hi[3] then a sequence of (rot, k); prints the decoded
    // cube after every step, then the 8 children of the last node and their flags
    Domain d;
    for (int k = 0; k < 3; ++k) scanf("%lf", &d.t_lo[k]);
    for (int k = 0; k < 3; ++k) scanf("%lf", &d.t_hi[k]);
    Node n;
    memset(&n, 0, sizeof n);
    n.flags = 1u;
    CubeGeom g;
    decode(n, d, g);
    put(g);
    int rot, k;
    while (scanf("%d %d", &rot, &k) == 2) {
        n = child_of(n, k, rot != 0);
        n.flags |= 1u;
        decode(n, d, g);
        put(g);
    }
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 8; ++c) {
            Node ch = child_of(n, c, r != 0);
            decode(ch, d, g);
            printf("child %d %d %u ", r, c, ch.flags & 1u);
            put(g);
        }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if not nvcc:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("branch")
    src, exe = d / "h.cu", d / "h"
    src.write_text(HARNESS)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC, str(src),
                    "-o", str(exe)], check=True, capture_output=True)
    return str(exe)


def _replay(t_lo, t_hi, path):
    """Sec. 4.1's split from the root [-pi, pi]^3 x [t_lo, t_hi], in FP64:
    a rotation split halves the rotation cube, a translation split the
    cuboid; child k takes the upper half along axis a when bit a of k is set."""
    r0, rhw = np.zeros(3), np.pi
    t0, thw = 0.5 * (np.array(t_lo) + np.array(t_hi)), 0.5 * (np.array(t_hi) - np.array(t_lo))
    out = [np.concatenate([r0, [rhw], t0, thw])]
    for rot, k in path:
        s = np.array([1.0 if (k >> a) & 1 else -1.0 for a in range(3)])
        if rot:
            rhw = rhw / 2
            r0 = r0 + s * rhw
        else:
            thw = thw / 2
            t0 = t0 + s * thw
        out.append(np.concatenate([r0, [rhw], t0, thw]))
    return np.array(out)


def _walk(exe, t_lo, t_hi, path):
    stdin = " ".join("%.17g" % v for v in list(t_lo) + list(t_hi)) + "\n"
    stdin += "\n".join("%d %d" % (r, k) for r, k in path) + "\n"
    out = subprocess.run([exe, "walk"], input=stdin, capture_output=True, text=True, check=True).stdout.splitlines()
    cubes = np.array([[float(v) for v in ln.split()] for ln in out if not ln.startswith("child")])
    kids = [ln.split()[1:] for ln in out if ln.startswith("child")]
    return cubes, [(int(a), int(b), int(c), np.array([float(v) for v in rest])) for a, b, c, *rest in kids]


def test_decoded_cells_follow_the_split(harness):
    rng = np.random.default_rng(0)
    for trial in range(40):
        t_lo = rng.uniform(-5, 0, 3)
        t_hi = t_lo + rng.uniform(0.5, 10, 3)
        path = [(int(rng.random() < 0.5), int(rng.integers(8))) for _ in range(int(rng.integers(0, 40)))]
        cubes, _ = _walk(harness, t_lo, t_hi, path)
        want = _replay(t_lo, t_hi, path)
        scale = np.concatenate([[np.pi] * 4, np.abs(t_lo) + np.abs(t_hi), np.abs(t_hi - t_lo)])
        assert cubes.shape == want.shape
        np.testing.assert_allclose(cubes, want, rtol=0, atol=1e-15 * scale.max() * 8)
        # half-widths are exact powers-of-two fractions of the root's
        np.testing.assert_array_equal(cubes[:, 3], want[:, 3])


def test_children_tile_the_parent(harness):
    rng = np.random.default_rng(1)
    for trial in range(20):
        t_lo, t_hi = np.array([-2.0, -1.5, -0.5]), np.array([2.0, 1.0, 3.0])
        path = [(int(rng.random() < 0.5), int(rng.integers(8))) for _ in range(int(rng.integers(0, 25)))]
        cubes, kids = _walk(harness, t_lo, t_hi, path)
        p = cubes[-1]
        for rot in (0, 1):
            ch = [c for r, k, f, c in kids if r == rot]
            flags = [f for r, k, f, c in kids if r == rot]
            assert len(ch) == 8
            # the self-sum cache survives a rotation split only
            assert flags == [1] * 8 if rot else flags == [0] * 8
            lo, hi = (0, 3) if rot else (4, 7)
            hw = (p[3:4] if rot else p[7:10]) / 2
            corners = set()
            for c in ch:
                np.testing.assert_array_equal(c[3:4] if rot else c[7:10], hw)
                keep = np.r_[4:10] if rot else np.r_[0:4]
                np.testing.assert_array_equal(c[keep], p[keep])  # the other part is untouched
                off = (c[lo:hi] - p[lo:hi]) / hw
                np.testing.assert_allclose(np.abs(off), 1.0, rtol=0, atol=1e-9)
                corners.add(tuple(np.sign(off).astype(int)))
            assert len(corners) == 8  # one child per octant: together they cover the parent exactly


def test_split_rule(harness):
    def rule(lr, lt, psit):
        out = subprocess.run([harness, "rule", str(lr), str(lt), "%.9g" % psit], capture_output=True, text=True,
                             check=True).stdout.split()
        return int(out[0]), float(out[1])
    # Lemma 2 with reading R1 at each level: min(sqrt(3) pi 2^-lr, pi)
    for lr in range(0, 12):
        assert rule(lr, 0, 0.0)[1] == pytest.approx(min(np.sqrt(3) * np.pi * 2.0 ** -lr, np.pi), rel=1e-15)
    # reading R6: split the rotation iff psi_r >= max psi_t (ties to rotation)
    psi3 = min(np.sqrt(3) * np.pi / 8, np.pi)
    assert rule(3, 2, psi3 * 0.999)[0] == 1
    assert rule(3, 2, psi3 * 1.001)[0] == 0
    below = np.float32(psi3)
    if below > psi3:
        below = np.nextafter(below, np.float32(0))
    assert rule(3, 2, float(below))[0] == 1  # the largest FP32 key at or below psi_r still splits the rotation
    # at every level the rule agrees with the FP64 comparison at the float
    # keys nearest psi_r (the kernels take it in FP32)
    for lr in range(0, 30):
        psi = min(np.sqrt(3) * np.pi * 2.0 ** -lr, np.pi)
        at = np.float32(psi)
        if float(at) > psi:
            at = np.nextafter(at, np.float32(0))
        for key in (at, np.nextafter(at, np.float32(np.inf)), np.nextafter(at, np.float32(0)), np.float32(0.0),
                    np.float32(4.0)):
            assert rule(lr, 0, float(key))[0] == int(psi >= float(key)), (lr, float(key))
    # level limits: a cell at the deepest level is never split further along that part
    assert rule(30, 5, 0.0)[0] == 0
    assert rule(5, 30, 10.0)[0] == 1


def test_priority_keys_order_like_their_floats(harness):
    rng = np.random.default_rng(2)
    vals = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000),
                           [-np.inf, -3.4e38, -1.0, -1e-40, -0.0, 0.0, 1e-40, 1.0, 3.4e38, np.inf]]).astype(np.float32)
    bits = vals.view(np.uint32)
    out = subprocess.run([harness, "keys"], input="\n".join("%x" % b for b in bits), capture_output=True, text=True,
                         check=True).stdout.split("\n")
    keys = np.array([int(ln.split()[0]) for ln in out if ln])
    back = np.array([int(ln.split()[1], 16) for ln in out if ln], dtype=np.uint32)
    np.testing.assert_array_equal(back, bits)  # the key decodes to the same float, bit for bit
    order = np.argsort(vals, kind="stable")
    v, k = vals[order], keys[order]
    strict = v[1:] > v[:-1]
    assert np.all(k[1:][strict] > k[:-1][strict])  # larger float, larger key
    assert np.all(k[1:] >= k[:-1])
    assert struct.unpack("<I", struct.pack("<f", -0.0))[0] != struct.unpack("<I", struct.pack("<f", 0.0))[0]
