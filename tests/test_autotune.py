"""Host logic of the schedule autotuner (no GPU): size classes, table lookup and the
fallback to the library defaults."""
from paper_2509_26581_gb300 import autotune


def test_size_classes():
    assert autotune.size_class(2_000) == "window"
    assert autotune.size_class(19_999) == "window"
    assert autotune.size_class(20_000) == "small"
    assert autotune.size_class(3_000_000) == "medium"
    assert autotune.size_class(29_000_000) == "large"


def test_choose_reads_the_table_and_falls_back():
    table = {"GPU X|ba|bf16|medium": {"best": {"chunk_edges": 256, "spmv_variant": 1}}}
    assert autotune.choose(3_000_000, "bf16", "ba", table, device="GPU X") == {"chunk_edges": 256, "spmv_variant": 1}
    assert autotune.choose(3_000_000, "fp64", "ba", table, device="GPU X") == autotune.DEFAULT
    assert autotune.choose(3_000_000, "bf16", "vi", table, device="GPU X") == autotune.DEFAULT
    assert autotune.choose(3_000_000, "bf16", "ba", table, device="GPU Y") == autotune.DEFAULT


def test_candidates_cover_the_three_kernels_and_three_chunk_sizes():
    assert {c["spmv_variant"] for c in autotune.CANDIDATES} == {1, 2, 3}
    assert {c["chunk_edges"] for c in autotune.CANDIDATES} == {256, 512, 1024}
    # the untuned default leaves the kernel choice to the library (automatic)
    assert autotune.DEFAULT == {"chunk_edges": 512, "spmv_variant": 0}
