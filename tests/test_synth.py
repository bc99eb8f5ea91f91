"""The seeded input generators (CPU only): determinism, ranges, and the
published SplitMix64 output they are built on."""
import numpy as np

import synth


def test_splitmix64_published_first_output():
    # SplitMix64 (Steele, Lea & Flood 2014) seeded with 0 first returns
    # 0xE220A8397B1DCDAF, the value of the published reference generator.
    assert synth.mix64(0) == 0xE220A8397B1DCDAF


def test_deterministic_and_thread_independent():
    a = synth.uniform(1 << 19, -5, 5, seed=3, tag=1)  # multi-threaded path
    b = synth.uniform(1 << 19, -5, 5, seed=3, tag=1)
    assert np.array_equal(a, b)
    small = synth.uniform(1000, -5, 5, seed=3, tag=1)  # single-threaded path
    assert np.array_equal(a[:1000], small)
    assert not np.array_equal(a, synth.uniform(1 << 19, -5, 5, seed=4, tag=1))


def test_uniform_ranges_inclusive():
    li = synth.lineitem(400_000, seed=1)
    expect = {"flag": (0, 2), "status": (0, 1), "qty": (1, 50), "price": (90000, 10500000),
              "disc": (0, 10), "tax": (0, 8), "date": (0, 2526)}
    for k, (lo, hi) in expect.items():
        assert li[k].min() >= lo and li[k].max() <= hi, k
        if hi - lo < 10_000:  # narrow ranges: both endpoints are drawn
            assert li[k].min() == lo and li[k].max() == hi, k
    assert li["flag"].dtype == np.uint8 and li["date"].dtype == np.int32
    # selectivity of date <= 2430 is 2431/2527
    sel = (li["date"] <= 2430).mean()
    assert abs(sel - 2431 / 2527) < 0.003


def test_join_build_distinct_and_in_range():
    k, p = synth.join_build(300_000, seed=2)
    assert len(np.unique(k)) == len(k)
    assert k.min() >= 0 and k.max() < (1 << 40)
    assert p.min() >= 0


def test_join_probe_absent_keys_really_absent():
    nb = 5000
    bk, _ = synth.join_build(nb, seed=4)
    pk, present = synth.join_probe(200_000, nb, seed=4)
    inb = np.isin(pk, bk)
    assert np.array_equal(inb, present.astype(bool))
    assert abs(present.mean() - 0.9) < 0.005


def test_zipf_head_probability_and_bounds():
    z = synth.Zipf(1000, 1.1)
    try:
        assert z.rank_of(0.0) == 1 and z.rank_of(1.0 - 2**-53) == 1000
        keys = z.keys(400_000, seed=1, mix=False)
        assert keys.min() >= 1 and keys.max() <= 1000
        h = sum(k ** -1.1 for k in range(1, 1001))
        for r in (1, 2, 10):
            p = (keys == r).mean()
            assert abs(p - r ** -1.1 / h) < 0.004, r
    finally:
        z.close()


def test_few_keys():
    k, v = synth.few_keys_kv(100_000, n_keys=4, seed=0)
    assert sorted(np.unique(k).tolist()) == sorted(synth.mix64_signed(i) for i in (1, 2, 3, 4))
    assert v.min() >= -1_000_000 and v.max() <= 1_000_000 and v.min() < -999_000


def test_gpu_instance_recipe_ranges():
    from synth import gpu as G

    fams = set()
    for seed in range(300):
        inst = G.instance(seed)
        assert 1_000_000 <= inst["rows"] <= 50_000_000
        assert 10 <= inst["domain"] <= 100_000_000
        fams.add(inst["family"])
        assert G.instance(seed) == inst
    assert fams == {f[0] for f in G.FAMILIES}


def test_batch_recipe_ranges_and_determinism():
    from synth import gpu as G

    r = G.batch_recipe(0)
    assert len(r["groupby"]) == 4096 and len(r["join"]) == 512
    rows = [x["rows"] for x in r["groupby"]]
    assert min(rows) >= 1000 and max(rows) <= 4_000_000
    assert all(1 <= x["groups"] <= 100_000 for x in r["groupby"])
    assert [x["key_type"] for x in r["groupby"][:4]] == ["int32", "int64", "int32", "int64"]
    assert all(1000 <= x["build"] <= 256_000 and 8000 <= x["probe"] <= 2_000_000
               for x in r["join"])
    # log-uniform rows: about 2e9 in all (mean (4e6 - 1e3) / ln 4000)
    assert 1.6e9 < sum(rows) < 2.4e9
    assert G.batch_recipe(0) == r and G.batch_recipe(1) != r
    seeds = [x["seed"] for x in r["groupby"]] + [x["seed"] for x in r["join"]]
    assert len(set(seeds)) == len(seeds)


def test_planner_instances_span_the_range():
    """The 32 planner-workload seeds the GPU oracle test checks
    (test_workload_oracle_gpu.py) cover the workload: small and large
    instances and every key family."""
    import synth.gpu

    insts = [synth.gpu.instance(s, rows_lo=1_000_000, rows_hi=50_000_000)
             for s in range(3_000_000, 3_000_032)]
    rows = [i["rows"] for i in insts]
    assert min(rows) < 3_000_000 and max(rows) > 25_000_000
    assert {i["family"] for i in insts} == {f[0] for f in synth.gpu.FAMILIES}
