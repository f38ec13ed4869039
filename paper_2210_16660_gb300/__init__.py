"""GB300-native PCG + aggregation-AMG pressure solver (arxiv 2210.16660 hot path)."""
