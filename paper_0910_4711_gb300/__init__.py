"""GB300-native LBG vector-quantizer design (Annaji & Rao, Sec. 2.2 / Alg. 1)."""
