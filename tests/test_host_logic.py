"""Host-side logic of the library that runs without a GPU, compiled with g++:
the semantic class layout (Sec. 4.2) that turns plain pair sums into the
weighted sum of the per-class objectives."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1812_01232_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include "classes.h"
// argv: nclass n1 n2, then n1c[nclass] n2c[nclass] w[nclass] phi1[n1] phi2[n2]
int main(int argc, char **argv) {
    int a = 1;
    const int nclass = atoi(argv[a++]), n1 = atoi(argv[a++]), n2 = atoi(argv[a++]);
    std::vector<int> n1c(nclass), n2c(nclass);
    std::vector<double> w(nclass), phi1(n1), phi2(n2);
    for (int l = 0; l < nclass; ++l) n1c[l] = atoi(argv[a++]);
    for (int l = 0; l < nclass; ++l) n2c[l] = atoi(argv[a++]);
    for (int l = 0; l < nclass; ++l) w[l] = atof(argv[a++]);
    for (int i = 0; i < n1; ++i) phi1[i] = atof(argv[a++]);
    for (int j = 0; j < n2; ++j) phi2[j] = atof(argv[a++]);
    gosma::ClassLayout L;
    const char *err = gosma::class_layout(nclass, n1c.data(), n2c.data(), w.data(), n1, n2, phi1.data(), phi2.data(), L);
    if (err) { printf("error %s\n", err); return 0; }
    printf("classes %d\n", (int)L.classes);
    for (int i = 0; i < n1; ++i) printf("row %.17g %d %d %d %d\n", L.phi1[i], L.cls1[i], L.rj0[i], L.rj1[i], L.rm1[i]);
    for (int j = 0; j < n2; ++j) printf("col %.17g %d\n", L.phi2[j], L.cls2[j]);
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("host")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _run(exe, n1c, n2c, w, phi1, phi2):
    args = [str(len(n1c)), str(len(phi1)), str(len(phi2))] + [str(v) for v in list(n1c) + list(n2c)]
    args += ["%.17g" % v for v in list(w) + list(phi1) + list(phi2)]
    out = subprocess.run([exe] + args, check=True, capture_output=True, text=True).stdout.split("\n")
    if out[0].startswith("error"):
        return out[0]
    rows = [l.split()[1:] for l in out if l.startswith("row")]
    cols = [l.split()[1:] for l in out if l.startswith("col")]
    return {"classes": int(out[0].split()[1]),
            "phi1": np.array([float(r[0]) for r in rows]), "cls1": [int(r[1]) for r in rows],
            "rj0": [int(r[2]) for r in rows], "rj1": [int(r[3]) for r in rows], "rm1": [int(r[4]) for r in rows],
            "phi2": np.array([float(c[0]) for c in cols]), "cls2": [int(c[1]) for c in cols]}


def test_one_class_changes_nothing(harness):
    phi1, phi2 = np.full(4, 0.25), np.array([0.5, 0.3, 0.2])
    r = _run(harness, [4], [3], [1.0], phi1, phi2)
    assert r["classes"] == 0
    np.testing.assert_array_equal(r["phi1"], phi1)
    np.testing.assert_array_equal(r["phi2"], phi2)
    assert r["rj0"] == [0] * 4 and r["rj1"] == [3] * 4 and r["rm1"] == [4] * 4


def test_classes_give_the_weighted_sum_of_class_pair_sums(harness):
    rng = np.random.default_rng(0)
    n1c, n2c, w = [2, 3, 1], [1, 2, 2], [0.25, 1.0, 4.0]
    phi1 = np.concatenate([rng.dirichlet(np.ones(a)) for a in n1c])
    phi2 = np.concatenate([rng.dirichlet(np.ones(b)) for b in n2c])
    r = _run(harness, n1c, n2c, w, phi1, phi2)
    assert r["classes"] == 1
    assert r["cls1"] == [0, 0, 1, 1, 1, 2] and r["cls2"] == [0, 1, 1, 2, 2]
    assert r["rj0"] == [0, 0, 1, 1, 1, 3] and r["rj1"] == [1, 1, 3, 3, 3, 5]
    assert r["rm1"] == [2, 2, 5, 5, 5, 6]
    # any pair term g: summing the scaled weights over within-class pairs gives sum_l w_l (class sum)
    g1 = rng.random((6, 6))
    g12 = rng.random((6, 5))
    s = sum(r["phi1"][i] * r["phi1"][m] * g1[i, m] for i in range(6) for m in range(6) if r["cls1"][i] == r["cls1"][m])
    c = sum(r["phi1"][i] * r["phi2"][j] * g12[i, j] for i in range(6) for j in range(r["rj0"][i], r["rj1"][i]))
    i0 = j0 = 0
    ref_s = ref_c = 0.0
    for l, (a, b) in enumerate(zip(n1c, n2c)):
        ii, jj = range(i0, i0 + a), range(j0, j0 + b)
        ref_s += w[l] * sum(phi1[i] * phi1[m] * g1[i, m] for i in ii for m in ii)
        ref_c += w[l] * sum(phi1[i] * phi2[j] * g12[i, j] for i in ii for j in jj)
        i0, j0 = i0 + a, j0 + b
    assert s == pytest.approx(ref_s, rel=1e-13) and c == pytest.approx(ref_c, rel=1e-13)


@pytest.mark.parametrize("n1c,n2c,w,phi1,phi2", [
    ([2, 2], [1, 1], [1.0, 1.0], [0.5, 0.5, 0.5, 0.4], [1.0, 1.0]),   # class weights do not sum to 1
    ([2, 1], [1, 1], [1.0, 1.0], [0.5, 0.5, 1.0, 1.0], [1.0, 1.0]),   # sizes do not add up to n1
    ([2, 2], [1, 1], [1.0, -1.0], [0.5, 0.5, 0.5, 0.5], [1.0, 1.0]),  # negative class weight
    ([2, 0], [1, 1], [1.0, 1.0], [0.5, 0.5], [1.0, 1.0]),             # empty class
])
def test_invalid_layouts_are_rejected(harness, n1c, n2c, w, phi1, phi2):
    assert str(_run(harness, n1c, n2c, w, phi1, phi2)).startswith("error")


RULES = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "host_rules.h"
int main(int argc, char **argv) {
    const char *what = argv[1];
    if (what[0] == 's') printf("%d\n", gosma::auto_pop_single(atoi(argv[2]), atoi(argv[3])));
    if (what[0] == 'b') printf("%d\n", gosma::auto_pop_batch(atoll(argv[2]), atoi(argv[3]), strtoull(argv[4], 0, 10)));
    if (what[0] == 'm') printf("%d\n", gosma::sma_block_for(atoi(argv[2]), atoi(argv[3]), atoi(argv[4]) != 0,
                                                            atoi(argv[5]), atoi(argv[6])));
    if (what[0] == 'p') {  // pick: ncand reps pref, then ncand * reps timings
        const int nc = atoi(argv[2]), reps = atoi(argv[3]), pref = atoi(argv[4]);
        std::vector<float> ms;
        for (int a = 5; a < argc; ++a) ms.push_back((float)atof(argv[a]));
        printf("%d\n", gosma::pick_shape(ms.data(), nc, reps, pref));
    }
    if (what[0] == 'q') {  // median: reps c, then the timings of the candidates
        const int reps = atoi(argv[2]), c = atoi(argv[3]);
        std::vector<float> ms;
        for (int a = 4; a < argc; ++a) ms.push_back((float)atof(argv[a]));
        printf("%d\n", (int)(1000.f * gosma::sample_median(ms.data(), c, reps) + 0.5f));
    }
    if (what[0] == 't') printf("%d\n", gosma::tune_stride(atoll(argv[2]), atoi(argv[3])));
    if (what[0] == 'r') printf("%d\n", gosma::retune_due(atoi(argv[2]), atoi(argv[3]), atoi(argv[4])) ? 1 : 0);
    if (what[0] == 'c') {  // candidates: wide group_bytes -> how many shapes
        gosma::BoundShape c[12];
        const int n = argc > 4 ? gosma::bound_shape_candidates(atoi(argv[2]), (size_t)atoll(argv[3]), c, atoi(argv[4]))
                               : gosma::bound_shape_candidates(atoi(argv[2]), (size_t)atoll(argv[3]), c);
        printf("%d\n", n);
    }
    if (what[0] == 'h') {  // hash: k, then values; the first k form one array, the rest another
        const int k = atoi(argv[2]);
        std::vector<double> v;
        for (int a = 3; a < argc; ++a) v.push_back(strtod(argv[a], 0));
        gosma::ProblemHash h;
        h.array(v.data(), (size_t)k);
        h.array(v.data() + k, v.size() - (size_t)k);
        printf("%lld\n", (long long)(h.h >> 1));
    }
    if (what[0] == 'f') {  // file skip count bytes: skip bytes, then ask for count records of bytes
        FILE *f = fopen(argv[2], "rb");
        if (!f) return 1;
        fseek(f, atol(argv[3]), SEEK_SET);
        bool ok = gosma::file_holds(f, strtoull(argv[4], 0, 10), strtoull(argv[5], 0, 10));
        printf("%d\n", ok ? (int)ftell(f) : -1 - (int)ftell(f));  // the position is kept either way
        fclose(f);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def rules(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("rules")
    src, exe = d / "r.cpp", d / "r"
    src.write_text(RULES)
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return lambda *a: int(subprocess.run([str(exe)] + [str(x) for x in a], check=True, capture_output=True,
                                          text=True).stdout)


def test_automatic_pop_of_one_problem(rules):
    assert rules("s", 10, 8) == 65536      # small mixtures: the most children per iteration
    assert rules("s", 128, 64) == 8192     # paper scale: 2^23 / 8192 = 1024, raised to the floor
    assert rules("s", 32, 32) == 8192      # 1024 pairs per cube
    assert rules("s", 16, 16) == 32768     # 2^23 / 256
    assert rules("s", 2048, 512) == 8192


def test_automatic_pop_of_a_batch(rules):
    assert rules("b", 80, 8, 1 << 26) == 65536
    assert rules("b", 256 * 128, 256, 1 << 18) == 256        # 2^23 / 32768
    assert rules("b", 80, 8, 1 << 18) == (1 << 18) // 16     # capacity / 16
    assert rules("b", 10 ** 7, 4, 1 << 26) == 64             # floor
    assert rules("b", 80, 60000, 1 << 26) == 0x7fffffff // (8 * 60000)  # 32-bit children offsets
    for nprob in (1, 7, 4096, 65535):
        assert 8 * rules("b", 80, nprob, 1 << 30) * nprob < 2 ** 31


def test_sma_threads_per_seed(rules):
    assert rules("m", 1, 152, 0, 128, 64) == 1024    # one large seed: a wide block
    assert rules("m", 1, 152, 1, 128, 64) == 512     # FP64 search: at most 512
    assert rules("m", 1, 152, 0, 10, 8) == 128       # 135 pair terms: no wider than 128
    assert rules("m", 1216, 152, 0, 128, 64) == 256  # 2048 x 152 / 1216 = 256 threads per seed
    assert rules("m", 4864, 152, 0, 128, 64) == 128


def test_checkpoint_reader_checks_the_file_size(rules, tmp_path):
    """file_holds: the records a checkpoint's header announces must be in the
    file before the reader sizes buffers from that count."""
    p = tmp_path / "ck.bin"
    p.write_bytes(bytes(1000))
    assert rules("f", p, 100, 900, 1) == 100          # exactly the rest of the file
    assert rules("f", p, 100, 13, 68) == 100          # 884 bytes of 900
    assert rules("f", p, 100, 14, 68) == -1 - 100     # 952 > 900: refused, position kept
    assert rules("f", p, 0, 0, 68) == 0
    assert rules("f", p, 0, 2 ** 62, 68) == -1        # the product would overflow: refused
    assert rules("f", p, 1000, 1, 1) == -1 - 1000     # nothing after the end


def test_checkpoint_problem_fingerprint(rules):
    """The fingerprint a checkpoint carries changes when any one mixture value
    changes, even by one unit in the last place, and when values move from one
    array to the next; equal arrays give equal fingerprints."""
    v = [0.25, -1.5, 3.0, 0.125, 2.0, 7.75]
    base = rules("h", 3, *["%.17g" % x for x in v])
    assert base == rules("h", 3, *["%.17g" % x for x in v])
    for i in range(len(v)):
        w = list(v)
        w[i] = float(np.nextafter(w[i], np.inf))
        assert rules("h", 3, *["%.17g" % x for x in w]) != base, i
    assert rules("h", 2, *["%.17g" % x for x in v]) != base
    assert rules("h", 4, *["%.17g" % x for x in v]) != base


def test_autotuner_picks_the_smallest_median(rules):
    """pick_shape on fake timing tables (3 timings per candidate): the
    smallest median wins, a single outlier does not decide, ties go to the
    earlier candidate, and a shape that could not run (1e30) never wins."""
    assert rules("p", 3, 3, -1, 2.0, 2.1, 1.9, 1.5, 1.6, 1.4, 1.7, 1.8, 1.6) == 1
    assert rules("p", 2, 3, -1, 1.0, 9.0, 1.1, 1.2, 1.2, 1.2) == 0      # median 1.1 beats 1.2 despite the 9.0
    assert rules("p", 2, 3, -1, 5.0, 0.1, 5.0, 1.0, 1.0, 1.0) == 1      # one fast outlier is not the median
    assert rules("p", 2, 3, -1, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0) == 0      # tie: the earlier candidate
    assert rules("p", 3, 3, -1, 1e30, 1e30, 1e30, 2.0, 2.0, 2.0, 1e30, 1e30, 1e30) == 1


def test_autotuner_keeps_the_default_within_the_margin(rules):
    """The default shape (pref) stays unless the winner's median is more
    than 3% below its own; a default that could not run never stays."""
    assert rules("p", 3, 3, 1, 0.98, 0.98, 0.98, 1.0, 1.0, 1.0, 1.2, 1.2, 1.2) == 1   # 2% faster: noise
    assert rules("p", 3, 3, 1, 0.96, 0.96, 0.96, 1.0, 1.0, 1.0, 1.2, 1.2, 1.2) == 0   # 4% faster: taken
    assert rules("p", 3, 3, 1, 1.1, 1.1, 1.1, 1.0, 1.0, 1.0, 1.2, 1.2, 1.2) == 1      # the default is best
    assert rules("p", 2, 3, 0, 1e30, 1e30, 1e30, 5.0, 5.0, 5.0) == 1


def test_sample_median(rules):
    """The median of one candidate's timings (in thousandths): odd and even
    counts, the other candidates' timings ignored."""
    assert rules("q", 3, 1, 9.0, 9.0, 9.0, 2.0, 1.0, 3.0) == 2000
    assert rules("q", 4, 0, 1.0, 4.0, 2.0, 3.0, 9.0, 9.0, 9.0, 9.0) == 2500


def test_autotuner_samples_a_sixteenth(rules):
    """Every stride-th run of four siblings: a sixteenth of the work, at
    least 64 children per SM, all of it for small iterations."""
    assert rules("t", 1 << 22, 152) == 16
    assert rules("t", 64 * 152 * 5, 152) == 5
    assert rules("t", 100, 152) == 1


def test_autotuner_retunes_when_half_the_problems_finished(rules):
    """retune_due(running at the last tuning, running now, iterations since):
    half the problems finished, some left, and at least 32 iterations since
    the last tuning (a short run would not earn the timings back)."""
    assert rules("r", 256, 128, 32) == 1 and rules("r", 256, 129, 32) == 0
    assert rules("r", 128, 64, 100) == 1 and rules("r", 1, 0, 100) == 0    # nothing left to tune for
    assert rules("r", 2, 1, 32) == 1
    assert rules("r", 256, 128, 31) == 0 and rules("r", 2, 1, 5) == 0      # too soon after the last tuning
    assert rules("r", 256, 256, 1000) == 0                                # nothing finished: no re-tuning


def test_autotuner_candidates(rules):
    """The shapes timed: a one-warp block only for tiny mixtures, wide blocks
    only where one problem would use them, no group narrower than a warp but
    the half-warp groups of 32x2 for mixtures of at most 16 model rows, and
    nothing whose groups' shared memory exceeds 200 KB per block."""
    assert rules("c", 32, 4096) == 9        # 32x1 64x1 64x2 128x1 128x2 128x4 256x1 256x2 256x4
    assert rules("c", 32, 4096, 16) == 10   # + 32x2
    assert rules("c", 32, 4096, 17) == 9
    assert rules("c", 128, 4096, 10) == 8   # no one-warp block for wider mixtures
    assert rules("c", 128, 4096) == 8       # no 32x1
    assert rules("c", 1024, 4096) == 9      # + 1024x1
    assert rules("c", 128, 60 * 1024) == 6  # 64x1 64x2 128x1 128x2 256x1 256x2: four groups of 60 KB do not fit
    assert rules("c", 512, 150 * 1024) == 4  # one group per block only: 64x1 128x1 256x1 512x1
