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


def test_autotuner_shape_and_group_choice_and_bracketing():
    """Block shape and launch-group budget are not semantic: the fastest wins, ties go to the
    candidate listed first; the round-count search reports whether its fastest candidate lies inside
    the range tried (bracketed) or at an end."""
    from paper_1701_04148_gb300 import autotune
    assert autotune.choose_fastest({512: 6.0, 256: 6.4, 128: 5.1}, (512, 256, 128)) == 256
    assert autotune.choose_fastest({512: 6.0, 256: 6.0, 128: 5.1}, (512, 256, 128)) == 512
    assert autotune.choose_fastest({None: 5.0, 1 << 26: 5.2, 0: 4.0}, [None, 1 << 26, 0]) == 1 << 26
    assert autotune.choose_fastest({None: 5.0, 0: 5.0}, [None, 0]) is None
    assert autotune.bracketed({8: 6.0, 16: 7.1, 32: 7.0, 64: 6.1})
    assert not autotune.bracketed({16: 6.0, 32: 7.1, 64: 6.1, 8: 7.2})
    assert not autotune.bracketed({8: 6.0, 16: 6.5, 1024: 6.6})
    assert autotune.ROUND_CANDIDATES[0] < 32 < autotune.ROUND_CANDIDATES[-1]
    assert set(autotune.BLOCK_CANDIDATES) == {512, 256, 128}


def test_kernel_source_hash_ignores_comments_only():
    """The bench keeps a committed traffic record only while the chunk kernels' code is unchanged:
    the hash drops comments and layout, keeps string literals (inline PTX) and every code token."""
    import bench
    strip = bench.code_without_comments
    a = 'int x = 1; // note\n/* block */ asm("ld.global.cg.u32 %0, [%1]; // not a comment");'
    b = 'int  x = 1;\n\n// other note\nasm("ld.global.cg.u32 %0, [%1]; // not a comment");  /* */'
    assert strip(a) == strip(b)
    assert "// not a comment" in strip(a)
    assert strip(a) != strip(a.replace("x = 1", "x = 2"))
    assert strip('char c = \'"\'; int y; // "') == 'char c = \'"\'; int y;'
    assert len(bench.chunk_kernel_source_sha256()) == 64


def test_autotune_cache_survives_a_bad_file(tmp_path):
    """The plan cache is read defensively (a missing, empty or half-written file means: tune again)
    and replaced atomically, since one process per GPU may tune at the same time."""
    from paper_1701_04148_gb300 import autotune
    p = tmp_path / "cache.json"
    assert autotune._read_cache(str(p)) == {}
    p.write_text('{"a": {"rounds": 4}')          # cut short
    assert autotune._read_cache(str(p)) == {}
    p.write_text('{"a": {"rounds": 4}}')
    assert autotune._read_cache(str(p)) == {"a": {"rounds": 4}}
