"""GB300-native vector order-statistic filters (VMF, BVDF, AMNFE/G, EVMF)
with exact and minimax elementary functions."""
