// push_menu.h -- the compiled (dimension, tile, drift) configurations of the
// particle kernel.  Each entry is instantiated for shape orders 1, 2 and 3.
//   2D: 16x16 tiles with drift 1, 2 (default) or 3; 8x8 with drift 1;
//       32x32 with drift 2.
//   3D: 8x8x8 tiles with drift 1 (default) or 2; 8x8x4 with drift 1 (small
//       enough for two 256-thread CTAs per SM).
#pragma once
#define PIC_PUSH_MENU_2D(X) X(16, 16, 1, 1) X(16, 16, 1, 2) X(16, 16, 1, 3) X(8, 8, 1, 1) X(32, 32, 1, 2)
#define PIC_PUSH_MENU_3D_A(X) X(8, 8, 8, 1)
#define PIC_PUSH_MENU_3D_B(X) X(8, 8, 8, 2) X(8, 8, 4, 1)
// 3D entries also compiled with TMA staging of the field tile
#define PIC_PUSH_MENU_3D_TMA(X) X(8, 8, 8, 1)
