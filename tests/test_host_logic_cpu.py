"""Host-side planning logic that needs no GPU: the batch autotuner's chunk sizes and choice."""
def test_autotuner_chunks_and_choice():
    """Chunk sizes spread each stream over about R rounds (ceil(N/R), clamped to [2, 2^20]), and
    the tuner keeps the largest R within the tolerance of the best throughput."""
    from paper_1701_04148_gb300 import autotune
    assert autotune.chunk_sizes([1, 64, 65, 10 ** 7, 10 ** 9], 64) == [2, 2, 2, 156250, 1 << 20]
    assert autotune.chunk_sizes([100, 101], 50) == [2, 3]
    res = {32: 7.0e9, 64: 6.8e9, 256: 4.4e9, 1024: 3.1e9}
    assert autotune.choose_rounds(res, 0.05) == 64      # 6.8 >= 0.95 * 7.0
    assert autotune.choose_rounds(res, 0.02) == 32
    assert autotune.choose_rounds(res, 0.60) == 1024
    k1 = autotune.shape_key([1024, 2048], [10, 20], 4, 16, 4)
    assert k1 == autotune.shape_key([1024, 2048], [10, 20], 4, 16, 4)
    assert k1 != autotune.shape_key([1024, 2048], [10, 21], 4, 16, 4)
