"""CPU oracle of the multi-scale fast MPV stereo matcher.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the matcher itself never does.
"""
